// apm_api.cu -- the C ABI of libapm (include/apm.h): context, hierarchy
// planning and validation, device arenas, and the per-level launch sequences.
#include <algorithm>
#include <climits>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "apm_internal.cuh"

using namespace apm;

namespace {

// NVTX range for the lifetime of the object: every API call and every kernel
// launch appears by name on a timeline tool's NVTX row (nvtx3 is header-only;
// with no tool attached each call returns at once)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

constexpr int kRoles = 11;
enum Role { R_GMF = 0, R_GAS, R_PGAS, R_GMF_IN, R_PHIS, R_PHIS_IN, R_PPHI, R_PACC, R_PHI, R_ACC, R_ACC_IN };
constexpr int kChunkCells = 2048;
constexpr double kPiHost = 3.141592653589793238462643383279502884;

// kernels, in launch order of one level
enum Kern { K_GAS = 0, K_DEPOSIT, K_XF, K_YF, K_Z, K_YI, K_XI, K_ACCEL, K_INTERP, K_ORDER, K_COUNT };
const char* const kKernelNames[K_COUNT] = {"gas_init", "tsc_deposit", "fft_x_fwd", "fft_y_fwd",
                                           "fft_z_green", "fft_y_inv", "fft_x_inv", "accel_carry",
                                           "tsc_interp", "particle_order"};

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;          // 2 per pair
    std::vector<int> kind;                // per used pair
    std::vector<int> n_launch;            // kernel launches inside each pair
    int used = 0;
    long long launches[K_COUNT] = {};
    double ms[K_COUNT] = {};
};

// Launch shape of one FFT pass over a level: the buffer budget that sets each
// grid's lines per CTA, the threads per CTA, and the resulting work list.
// One launch of a pass: a contiguous range of the work list whose grids all
// run the same kernel (fast_L = 0: the runtime-planned kernel; otherwise the
// FP32 kernel with the compile-time plan of that length).
struct PassSeg {
    int first = 0, count = 0;
    int fast_L = 0;
    size_t smem = 0;
};
struct PassPlan {
    int budget = 0;
    int threads = 0;
    Chunk* d = nullptr;
    int n = 0;
    std::vector<int> lines;          // per grid of the level
    std::vector<int> first, count;   // per grid: its chunks [first, first + count)
    std::vector<int> seg_of;         // per grid: its segment
    std::vector<PassSeg> seg;
};

struct Level {
    int level = 0;
    std::vector<int> grids;          // hierarchy indices, in order
    std::vector<GridDev> hg;         // host copies of the descriptors
    GridDev* d_grids = nullptr;
    LevelDev dev{};
    // CTA work lists: the FFT passes (launch shape per pass), baryons, accelerations
    PassPlan pass[kFftPasses];
    // autotuned plan choices (apm_fft_shapes): per pass, the compile-time plan
    // where a length has one (0) or the runtime plan (1); the runtime plans'
    // largest stage radix; the order grids are packed into each work list
    int plan[kFftPasses] = {0, 0, 0, 0, 0};
    int max_radix = 16;
    int packing = 0;                 // 0 hierarchy order, 1 largest transform first
    Chunk* d_gas = nullptr; int n_gas = 0;
    Chunk* d_acc = nullptr; int n_acc = 0;
    std::vector<int> acc_first;      // per grid: its first acceleration chunk (ng + 1 entries)
    // pointer tables (device) + pinned mirrors + last uploaded values
    int cap = 0;
    void** d_ptr = nullptr;          // kRoles * cap
    void** h_ptr = nullptr;          // pinned, kRoles * cap
    std::vector<void*> last[kRoles];
    cudaEvent_t ev = nullptr;
    bool ev_pending = false;
};

}  // namespace

struct apm_ctx {
    apm_config cfg{};
    int device = 0;
    unsigned* d_status = nullptr;
    bool has_hier = false;
    std::vector<apm_grid> grids;
    std::vector<int> level_of, index_in_level;
    std::vector<Level> levels;
    std::vector<void*> dev_allocs;
    double2* tw64 = nullptr;
    float2* tw32 = nullptr;
    double* tab64 = nullptr;
    float* tab32 = nullptr;
    void* wsA = nullptr;
    void* wsB = nullptr;
    void* wsC = nullptr;             // spectral gradient: the y-inverse output, so wsB keeps the forward
    LevelDev* d_levels = nullptr;    // every level's LevelDev (the all-level kernels)
    void** d_tabs = nullptr;         // [role][level]: each level's device pointer table of the role
    Profiler prof;
    bool batched = true;             // apm_set_grid_batching
    bool dep_tiles = false;          // apm_set_deposit_tiles
    // auxiliary streams on which the segments of one FFT pass (grids of
    // different kernels) run side by side, forked from and joined to the
    // caller's stream with events
    static constexpr int kAux = 3;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kAux] = {};
    std::vector<cudaGraphExec_t> graphs;   // apm_graph_end (null: destroyed)
    // particle processing order (apm_reserve_order / apm_order_particles)
    struct Order {
        long long cap = 0;           // particles the workspace holds (0: no ordering)
        int shift = 0, nb = 0;       // bins: cubes of 2^shift root cells, nb per axis
        unsigned *count = nullptr, *sums = nullptr, *key = nullptr, *rank = nullptr;
        int* perm = nullptr;
        long long n = -1;            // particle count of the current order (-1: none)
    } order;
};

namespace {

bool fault_alloc() {
    const char* f = std::getenv("APM_FAULT_INJECT");
    return f && std::strcmp(f, "alloc") == 0;
}

// APM_FAULT_INJECT=wait: the x-forward pass's bulk copy waits for 16 bytes
// more than it copies, so its bounded mbarrier wait runs out (tests the
// timeout path; nothing faults)
bool fault_wait() {
    const char* f = std::getenv("APM_FAULT_INJECT");
    return f && std::strcmp(f, "wait") == 0;
}

apm_status dmalloc(apm_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (fault_alloc()) return APM_E_NOMEM;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? APM_E_NOMEM : APM_E_CUDA;
    }
    c->dev_allocs.push_back(*p);
    return APM_OK;
}

template <typename V>
apm_status upload(apm_ctx* c, V** dst, const std::vector<V>& src) {
    apm_status st = dmalloc(c, (void**)dst, src.size() * sizeof(V));
    if (st != APM_OK) return st;
    if (!src.empty() &&
        cudaMemcpy(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice) != cudaSuccess)
        return APM_E_CUDA;
    return APM_OK;
}

void dfree(apm_ctx* c, void* p) {
    if (!p) return;
    cudaFree(p);
    auto it = std::find(c->dev_allocs.begin(), c->dev_allocs.end(), p);
    if (it != c->dev_allocs.end()) c->dev_allocs.erase(it);
}

void free_graphs(apm_ctx* c) {
    for (cudaGraphExec_t g : c->graphs)
        if (g) cudaGraphExecDestroy(g);
    c->graphs.clear();
}

void free_hierarchy(apm_ctx* c) {
    cudaDeviceSynchronize();
    free_graphs(c);   // they replay launches on the buffers freed below
    for (void* p : c->dev_allocs) cudaFree(p);
    c->dev_allocs.clear();
    for (Level& L : c->levels) {
        if (L.h_ptr) cudaFreeHost(L.h_ptr);
        if (L.ev) cudaEventDestroy(L.ev);
    }
    c->levels.clear();
    c->grids.clear();
    c->level_of.clear();
    c->index_in_level.clear();
    c->tw64 = nullptr; c->tw32 = nullptr; c->tab64 = nullptr; c->tab32 = nullptr;
    c->wsA = nullptr; c->wsB = nullptr; c->wsC = nullptr;
    c->d_levels = nullptr; c->d_tabs = nullptr;
    c->order = apm_ctx::Order();     // its arrays were among dev_allocs
    c->has_hier = false;
}

int smooth7_at_least(int n) {
    for (int m = std::max(n, 1);; ++m) {
        int r = m;
        for (int p : {2, 3, 5, 7})
            while (r % p == 0) r /= p;
        if (r == 1) return m;
    }
}

// the isolated root's transform length with the four-point gradient: even, and
// at least 2 N + 2 so that phi at cells -2 and N + 1 (read by the stencils of
// the edge cells) sees every mass at its true offset
int even_smooth7_at_least(int n) {
    int m = smooth7_at_least(n);
    while (m & 1) m = smooth7_at_least(m + 1);
    return m;
}

long long floor_div(long long a, long long b) {
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// the FP32 column passes use the compile-time plans of fft_fast.cuh where a
// length has one (APM_FFT_FAST=0 keeps every pass on the runtime-planned
// kernels, for comparison)
bool fft_fast_enabled() {
    const char* v = std::getenv("APM_FFT_FAST");
    return !(v && std::atoi(v) == 0);
}

// largest FFT stage radix of the FP32 path (16; APM_FFT_MAX_RADIX overrides it,
// 8 restricts the plans to the simple radices)
int fft_max_radix() {
    const char* e = std::getenv("APM_FFT_MAX_RADIX");
    int v = e ? std::atoi(e) : 16;
    return v < 8 ? 8 : (v > 16 ? 16 : v);
}

int border_cells(const apm_config& c) {
    return (int)std::ceil(c.pad_factor * c.refine * c.a_over_dx - 1e-12);
}

// Validates the tree (see apm_set_hierarchy).
apm_status validate(const apm_config& cfg, const apm_grid* gr, int n) {
    if (n < 1) return APM_E_INVALID;
    const apm_grid& r = gr[0];
    if (r.level != 0 || r.parent != -1 || r.start[0] || r.start[1] || r.start[2]) return APM_E_NESTING;
    if (r.dims[0] != r.dims[1] || r.dims[0] != r.dims[2] || r.dims[0] < 4) return APM_E_INVALID;
    int maxlev = 0;
    for (int i = 1; i < n; ++i) {
        const apm_grid& g = gr[i];
        if (g.level < 1 || g.parent < 0 || g.parent >= n || g.parent == i) return APM_E_NESTING;
        if (gr[g.parent].level != g.level - 1) return APM_E_NESTING;
        for (int j = 0; j < 3; ++j)
            if (g.dims[j] < 1) return APM_E_INVALID;
        maxlev = std::max(maxlev, g.level);
    }
    std::vector<int> count(maxlev + 1, 0);
    for (int i = 0; i < n; ++i) {
        if (gr[i].level == 0 && i != 0) return APM_E_NESTING;
        count[gr[i].level]++;
    }
    for (int l = 0; l <= maxlev; ++l)
        if (count[l] == 0) return APM_E_NESTING;
    const int R = cfg.refine;
    const int B = border_cells(cfg);
    for (int i = 1; i < n; ++i) {
        const apm_grid& g = gr[i];
        const apm_grid& p = gr[g.parent];
        // nothing lies outside an isolated root: the GMF border of its children
        // may extend past it (those baryons are zero); the carry may not
        const bool past_root = g.parent == 0 && cfg.root_bc == APM_BC_ISOLATED;
        for (int j = 0; j < 3; ++j) {
            // parent cells read by the GMF border (baryons) and by the carry of cells [-1, N]
            long long lo_b = floor_div(g.start[j] - B, R);
            long long hi_b = floor_div(g.start[j] + g.dims[j] + B - 1, R);
            long long lo_c = (long long)std::floor((g.start[j] - 1 + 0.5) / R - 0.5);
            long long hi_c = (long long)std::floor((g.start[j] + g.dims[j] + 0.5) / R - 0.5) + 1;
            long long lo = past_root ? lo_c : std::min(lo_b, lo_c);
            long long hi = past_root ? hi_c : std::max(hi_b, hi_c);
            if (lo < p.start[j] || hi >= p.start[j] + p.dims[j]) return APM_E_NESTING;
        }
    }
    for (int i = 1; i < n; ++i)
        for (int k = i + 1; k < n; ++k) {
            if (gr[i].level != gr[k].level) continue;
            bool overlap = true;
            for (int j = 0; j < 3; ++j)
                if (!(gr[i].start[j] < gr[k].start[j] + gr[k].dims[j] &&
                      gr[k].start[j] < gr[i].start[j] + gr[i].dims[j]))
                    overlap = false;
            if (overlap) return APM_E_NESTING;
        }
    return APM_OK;
}

// CSR of the grids whose box [lo, hi) (level cells) meets each tile
void build_csr(const std::vector<std::pair<std::array<long long, 3>, std::array<long long, 3>>>& boxes,
               const long long mlo[3], int shift, const int nt[3], std::vector<int>& off,
               std::vector<int>& list) {
    long long ntiles = (long long)nt[0] * nt[1] * nt[2];
    std::vector<std::vector<int>> per(ntiles);
    for (size_t gi = 0; gi < boxes.size(); ++gi) {
        long long t0[3], t1[3];
        bool empty = false;
        for (int j = 0; j < 3; ++j) {
            long long a = boxes[gi].first[j] - mlo[j], b = boxes[gi].second[j] - mlo[j] - 1;
            a = std::max(a, 0LL);
            b = std::min(b, ((long long)nt[j] << shift) - 1);
            if (b < a) empty = true;
            t0[j] = a >> shift;
            t1[j] = b >> shift;
        }
        if (empty) continue;
        for (long long z = t0[2]; z <= t1[2]; ++z)
            for (long long y = t0[1]; y <= t1[1]; ++y)
                for (long long x = t0[0]; x <= t1[0]; ++x)
                    per[x + nt[0] * (y + (long long)nt[1] * z)].push_back((int)gi);
    }
    off.assign(ntiles + 1, 0);
    list.clear();
    for (long long t = 0; t < ntiles; ++t) {
        off[t] = (int)list.size();
        list.insert(list.end(), per[t].begin(), per[t].end());
    }
    off[ntiles] = (int)list.size();
}

apm_status cuda_status(cudaError_t e) { return e == cudaSuccess ? APM_OK : APM_E_CUDA; }

// Work list of FFT pass q over the grids of a level for a buffer budget and a
// CTA size: each grid's lines per CTA (halved until the CTA fits its shared
// memory), one chunk per CTA.  The lines batch whole lines, so the shape never
// changes a result.
apm_status build_pass(apm_ctx* c, const Level& L, int q, int budget, int threads, bool f64, PassPlan& P) {
    const size_t csz = f64 ? sizeof(double2) : sizeof(float2);
    const int ng = (int)L.hg.size();
    std::vector<Chunk> list;
    P.lines.assign(ng, 0);
    P.first.assign(ng, 0);
    P.count.assign(ng, 0);
    P.seg_of.assign(ng, 0);
    P.seg.clear();
    // the kernel of each grid: a compile-time plan for the FP32 passes of its
    // length, if there is one (not for the x-forward pass while its bulk-copy
    // wait is made to run out); a spectral gradient's components run the z pass
    // on the same work list (k_col_fast MODE 3, or k_col MODE 3)
    std::vector<int> fast(ng, 0), lens(ng, 0);
    const bool row = q == kPassXf || q == kPassXi;
    // with plan 2 on the x-forward pass, a grid with M0 = M1 whose plane fits
    // runs the fused x + y forward (k_xy_fast) as its x-forward segment (kind
    // -L) and has no y-forward work (kind kSkip); other grids run plan 0
    constexpr int kSkip = INT_MIN;
    // (the kernel stores row pair p in plane rows 2p, 2p + 1: an odd G1 needs
    // G1 < M1, so that the pairs fit the M1 rows of the plane)
    auto fused_xy = [&](const GridDev& g) {
        return !f64 && L.plan[kPassXf] == 2 && fft_fast_enabled() && !fault_wait() && g.M[0] == g.M[1] &&
               fast_xy_length(g.M[0]) && 2 * ((g.G[1] + 1) / 2) <= g.M[1];
    };
    // ... and the fused y + x inverse (k_yx_fast) as its x-inverse segment when
    // the window's row pairs are distinct rows of the transform (2 ceil(W1/2)
    // <= M1: a periodic root, whose window is taller than M1, is excluded)
    auto fused_yx = [&](const GridDev& g) {
        return !f64 && L.plan[kPassXi] == 2 && fft_fast_enabled() && g.M[0] == g.M[1] && fast_xy_length(g.M[0]) &&
               2 * ((g.W[1] + 1) / 2) <= g.M[1];
    };
    for (int k = 0; k < ng; ++k) {
        const GridDev& g = L.hg[k];
        lens[k] = row ? g.M[0] : (q == kPassZ ? g.M[2] : g.M[1]);
        if (!f64 && L.plan[q] != 1 && fft_fast_enabled() && fast_length(lens[k]) &&
            !(q == kPassXf && fault_wait()))
            fast[k] = lens[k];
        if ((q == kPassXf || q == kPassYf) && fused_xy(g)) fast[k] = q == kPassXf ? -lens[k] : kSkip;
        if ((q == kPassXi || q == kPassYi) && fused_yx(g)) fast[k] = q == kPassXi ? -lens[k] : kSkip;
    }
    std::vector<int> kinds(fast);
    std::sort(kinds.begin(), kinds.end());
    kinds.erase(std::unique(kinds.begin(), kinds.end()), kinds.end());
    // packing: the order of the grids inside each segment's work list
    std::vector<int> order(ng);
    for (int k = 0; k < ng; ++k) order[k] = k;
    if (L.packing == 1) {
        auto work = [&](int k) { return (long long)L.hg[k].M[0] * L.hg[k].M[1] * L.hg[k].M[2]; };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
    }
    for (int kind : kinds) {
        if (kind == kSkip) {            // fused into the x-forward segment: no chunks
            for (int k = 0; k < ng; ++k)
                if (fast[k] == kSkip) {
                    P.lines[k] = kFastTx;
                    P.first[k] = 0;
                    P.count[k] = 0;
                    P.seg_of[k] = 0;
                }
            continue;
        }
        PassSeg sg;
        sg.first = (int)list.size();
        sg.fast_L = kind;
        for (int k : order) {
            if (fast[k] != kind) continue;
            const GridDev& g = L.hg[k];
            const int len = lens[k];
            if (kind < 0) {             // fused x + y passes: one chunk per z (window) plane
                P.lines[k] = kFastNp;
                P.first[k] = (int)list.size();
                P.seg_of[k] = (int)P.seg.size();
                sg.smem = fast_xy_smem(len);
                const int planes = q == kPassXf ? g.G[2] : g.W[2];
                for (int zp = 0; zp < planes; ++zp) list.push_back({k, zp});
                P.count[k] = (int)list.size() - P.first[k];
                continue;
            }
            int lines;
            if (kind) {
                lines = row ? kFastNp : kFastTx;
                sg.smem = row ? fast_row_smem(len) : fast_col_smem(len);
            } else {
                lines = fft_pass_lines(q, len, budget, f64);
                while (lines > 1 && fft_pass_smem(q, len, lines, csz, g.G[0]) > (size_t)kFftSmemLimit) lines /= 2;
                sg.smem = std::max(sg.smem, fft_pass_smem(q, len, lines, csz, g.G[0]));
            }
            P.lines[k] = lines;
            P.first[k] = (int)list.size();
            P.seg_of[k] = (int)P.seg.size();
            if (q == kPassXf || q == kPassXi) {
                const long long rows = q == kPassXf ? (long long)g.G[1] * g.G[2] : (long long)g.W[1] * g.W[2];
                const long long n = ((rows + 1) / 2 + lines - 1) / lines;
                for (long long t = 0; t < n; ++t) list.push_back({k, (int)t});
            } else {
                // (kx tile, z | ky | zw) pairs, encoded as (kt << kColOtherBits) | other
                const int nkt = (g.Hx + lines - 1) / lines;
                const int n_other = q == kPassYf ? g.G[2] : (q == kPassZ ? g.M[1] : g.W[2]);
                for (int o = 0; o < n_other; ++o)
                    for (int kt = 0; kt < nkt; ++kt) list.push_back({k, (kt << kColOtherBits) | o});
            }
            P.count[k] = (int)list.size() - P.first[k];
        }
        sg.count = (int)list.size() - sg.first;
        P.seg.push_back(sg);
    }
    P.budget = budget;
    P.threads = threads;
    P.n = (int)list.size();
    P.d = nullptr;
    return upload(c, &P.d, list);
}

// copies pass q's lines per CTA into the host descriptors of the level
void apply_pass(Level& L, int q) {
    for (size_t k = 0; k < L.hg.size(); ++k) L.hg[k].lines[q] = L.pass[q].lines[k];
}

// the runtime plans of every grid of the level with stage radices up to r
// (FP32: 16 or 8; FP64 plans keep radices up to 8)
bool replan_level(Level& L, int r) {
    for (GridDev& g : L.hg) {
        FftPlan1D* pls[3] = {&g.fx, &g.fy, &g.fz};
        for (int j = 0; j < 3; ++j) {
            const int off = pls[j]->tw_off;
            if (!fft_plan(g.M[j], r, pls[j])) return false;
            pls[j]->tw_off = off;
        }
        fft_plan_reversed(g.fy, &g.iy);
        fft_plan_reversed(g.fz, &g.iz);
    }
    L.max_radix = r;
    return true;
}

// One launch of pass q over the chunks [first, first + count) of segment sg.
// comp: with the spectral gradient, the component (0 phi, 1-3 A_x..A_z) of
// the z, y-inverse and x-inverse passes; the y inverse then writes wsC, so
// the y-forward output in wsB stays for the next component's z pass.
cudaError_t run_seg(apm_ctx* c, const Level& L, int q, const PassPlan& P, const PassSeg& sg, int first, int count,
                    void** d_gmf, void** d_phis, cudaStream_t s, int comp) {
    const bool f64 = c->cfg.precision == APM_FP64;
    FftArgs a;
    a.g = L.d_grids;
    a.tw = f64 ? (const void*)c->tw64 : (const void*)c->tw32;
    a.tab = f64 ? (const void*)c->tab64 : (const void*)c->tab32;
    a.wsA = c->wsA;
    a.wsB = c->wsB;
    a.F = c->cfg.mass_frac_bits;
    a.chunks = P.d + first;
    a.n_chunks = count;
    a.smem = sg.smem;
    a.threads = P.threads;
    a.status = c->d_status;
    a.inject_wait = fault_wait() ? 1 : 0;
    a.comp = comp;
    if (c->cfg.gradient == APM_GRAD_SPECTRAL && (q == kPassYi || q == kPassXi)) a.wsB = c->wsC;
    if (sg.fast_L < 0)
        return q == kPassXf ? launch_fft_xy_fast(-sg.fast_L, a, (const int64_t* const*)d_gmf, s)
                            : launch_fft_yx_fast(-sg.fast_L, a, d_phis, s);
    if (sg.fast_L) {
        switch (q) {
            case kPassYf: return launch_fft_yf_fast(sg.fast_L, a, s);
            case kPassZ:   // component comp > 0 of a spectral gradient: the table times -i D_comp
                return comp > 0 ? launch_fft_zgrad_fast(sg.fast_L, a, s) : launch_fft_z_fast(sg.fast_L, a, s);
            case kPassYi: return launch_fft_yi_fast(sg.fast_L, a, s);
            case kPassXf: return launch_fft_xf_fast(sg.fast_L, a, (const int64_t* const*)d_gmf, s);
            default: return launch_fft_xi_fast(sg.fast_L, a, d_phis, s);
        }
    }
    switch (q) {
        case kPassXf:
            return f64 ? launch_fft_xf<double>(a, (const int64_t* const*)d_gmf, s)
                       : launch_fft_xf<float>(a, (const int64_t* const*)d_gmf, s);
        case kPassYf: return f64 ? launch_fft_yf<double>(a, s) : launch_fft_yf<float>(a, s);
        case kPassZ:
            if (comp > 0) return f64 ? launch_fft_zgrad<double>(a, s) : launch_fft_zgrad<float>(a, s);
            return f64 ? launch_fft_z<double>(a, s) : launch_fft_z<float>(a, s);
        case kPassYi: return f64 ? launch_fft_yi<double>(a, s) : launch_fft_yi<float>(a, s);
        default: return f64 ? launch_fft_xi<double>(a, d_phis, s) : launch_fft_xi<float>(a, d_phis, s);
    }
}

// launches FFT pass q of a level with plan P: every segment, or with grid >= 0
// only that grid's chunks (one grid's launch of the pass)
cudaError_t run_pass(apm_ctx* c, const Level& L, int q, const PassPlan& P, void** d_gmf, void** d_phis,
                     cudaStream_t s, int comp = 0, int grid = -1) {
    if (grid >= 0) {
        if (P.count[grid] == 0) return cudaSuccess;   // fused into another pass
        const PassSeg& sg = P.seg[P.seg_of[grid]];
        return run_seg(c, L, q, P, sg, P.first[grid], P.count[grid], d_gmf, d_phis, s, comp);
    }
    const int nseg = (int)P.seg.size();
    if (nseg <= 1) return nseg ? run_seg(c, L, q, P, P.seg[0], P.seg[0].first, P.seg[0].count, d_gmf, d_phis, s, comp)
                               : cudaSuccess;
    // the segments write disjoint grids: segment 0 on the caller's stream, the
    // others round-robin on the auxiliary streams, so that one segment's last
    // partial wave overlaps the next one's CTAs
    const int used = std::min(nseg - 1, apm_ctx::kAux);
    cudaError_t e = cudaEventRecord(c->ev_fork, s);
    for (int j = 0; j < used && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(c->aux[j], c->ev_fork, 0);
    for (int i = 0; i < nseg && e == cudaSuccess; ++i) {
        const PassSeg& sg = P.seg[i];
        e = run_seg(c, L, q, P, sg, sg.first, sg.count, d_gmf, d_phis, i == 0 ? s : c->aux[(i - 1) % used], comp);
    }
    // joined even after a failed launch, so that no auxiliary stream stays
    // forked from a capturing stream
    for (int j = 0; j < used; ++j) {
        const cudaError_t e1 = cudaEventRecord(c->ev_join[j], c->aux[j]);
        const cudaError_t e2 = cudaStreamWaitEvent(s, c->ev_join[j], 0);
        if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    }
    return e;
}

// Uploads the device pointers of one role if they changed since the last call.
apm_status set_ptrs(apm_ctx* c, Level& L, int role, const void* const* host, int count,
                    void*** dev_out, cudaStream_t s) {
    *dev_out = nullptr;
    if (!host) return APM_OK;
    if (count > L.cap) return APM_E_INVALID;
    std::vector<void*>& last = L.last[role];
    bool same = (int)last.size() == count;
    for (int i = 0; same && i < count; ++i) same = last[i] == host[i];
    void** dev = L.d_ptr + (size_t)role * L.cap;
    if (!same) {
        if (L.ev_pending) {
            if (cudaEventSynchronize(L.ev) != cudaSuccess) return APM_E_CUDA;
            L.ev_pending = false;
        }
        void** h = L.h_ptr + (size_t)role * L.cap;
        for (int i = 0; i < count; ++i) h[i] = const_cast<void*>(host[i]);
        if (cudaMemcpyAsync(dev, h, count * sizeof(void*), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return APM_E_CUDA;
        if (cudaEventRecord(L.ev, s) != cudaSuccess) return APM_E_CUDA;
        L.ev_pending = true;
        last.resize(count);
        for (int i = 0; i < count; ++i) last[i] = const_cast<void*>(host[i]);
    }
    *dev_out = dev;
    return APM_OK;
}

// brackets one launch with events when tracing is on
struct Trace {
    apm_ctx* c;
    int pair = -1;
    cudaStream_t s;
    Range range;
    Trace(apm_ctx* ctx, int k, cudaStream_t st) : c(ctx), s(st), range(kKernelNames[k]) {
        Profiler& P = c->prof;
        if (!P.on || P.used * 2 + 1 >= (int)P.ev.size()) return;
        pair = P.used++;
        P.kind[pair] = k;
        P.n_launch[pair] = 1;
        cudaEventRecord(P.ev[2 * pair], s);
    }
    // the bracket holds n launches of the kernel (an FFT pass of several segments)
    void launches(int n) {
        if (pair >= 0) c->prof.n_launch[pair] = n;
    }
    ~Trace() {
        if (pair >= 0) cudaEventRecord(c->prof.ev[2 * pair + 1], s);
    }
};

void profile_free(Profiler& P) {
    for (cudaEvent_t e : P.ev) cudaEventDestroy(e);
    P.ev.clear();
    P.kind.clear();
    P.used = 0;
    P.on = false;
}

Particles to_dev(const apm_particles* p) {
    Particles q;
    q.n = p->n;
    q.x = p->x; q.y = p->y; q.z = p->z;
    q.vx = p->vx; q.vy = p->vy; q.vz = p->vz;
    q.m = p->m;
    return q;
}

// the interpolation calls visit the particles in the current order when it
// was computed for this many particles (any order gives the same results);
// so do the deposits with apm_set_deposit_tiles(1), which then gather each
// CTA's charges of its bin in shared memory (k_deposit<true>).  Without the
// tiles the deposits keep the caller's order: in bin order neighbouring
// threads reduce into the same cells and their L2 reductions serialise.
void use_order(const apm_ctx* c, Particles& P) {
    if (c->order.perm && c->order.n == P.n) {
        P.perm = c->order.perm;
        P.order_shift = c->order.shift;
    }
}

bool particles_ok(const apm_particles* p) {
    if (!p || p->n < 0) return false;
    if (p->n == 0) return true;
    return p->x && p->y && p->z && p->vx && p->vy && p->vz && p->m;
}

}  // namespace

extern "C" {

void apm_config_default(apm_config* cfg) {
    if (!cfg) return;
    cfg->box = 1.0;
    cfg->a_over_dx = 3.4;
    cfg->refine = 2;
    cfg->pad_factor = 0.65;
    cfg->root_bc = APM_BC_ISOLATED;
    cfg->precision = APM_FP32;
    cfg->mass_frac_bits = 52;
    cfg->root_correction = 1;
    cfg->device = -1;
    cfg->gradient = APM_GRAD_FD2;
}

const char* apm_version(void) { return "apm-gb300 0.1 (sm_103a)"; }

const char* apm_status_string(apm_status s) {
    switch (s) {
        case APM_OK: return "ok";
        case APM_E_INVALID: return "invalid argument";
        case APM_E_NESTING: return "hierarchy violates the nesting rules";
        case APM_E_NOMEM: return "out of memory";
        case APM_E_CUDA: return "CUDA runtime error";
        case APM_E_OVERFLOW: return "fixed-point overflow (particle skipped)";
        case APM_E_OUT_OF_BOX: return "particle outside the isolated root (folded)";
        case APM_E_TIMEOUT: return "device wait ran out";
        case APM_E_UNSUPPORTED: return "unsupported request";
        case APM_E_STATE: return "call out of order";
        case APM_E_BOUNDS: return "device access out of range (bounds-checked build)";
    }
    return "unknown status";
}

apm_status apm_create(const apm_config* cfg, apm_ctx** out) {
    if (!cfg || !out) return APM_E_INVALID;
    *out = nullptr;
    if (!(cfg->box > 0) || !(cfg->a_over_dx > 0) || cfg->refine < 2 || !(cfg->pad_factor >= 0) ||
        (cfg->root_bc != APM_BC_ISOLATED && cfg->root_bc != APM_BC_PERIODIC) ||
        (cfg->precision != APM_FP32 && cfg->precision != APM_FP64) || cfg->mass_frac_bits < 1 ||
        cfg->mass_frac_bits > 62 ||
        (cfg->gradient != APM_GRAD_FD2 && cfg->gradient != APM_GRAD_FD4 && cfg->gradient != APM_GRAD_SPECTRAL))
        return APM_E_INVALID;
    if (cfg->refine != 2) return APM_E_UNSUPPORTED;
    apm_ctx* c = new apm_ctx();
    c->cfg = *cfg;
    if (cfg->device >= 0 && cudaSetDevice(cfg->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return APM_E_CUDA;
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return APM_E_CUDA;
    }
    bool aux_ok = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int j = 0; j < apm_ctx::kAux && aux_ok; ++j)
        aux_ok = cudaStreamCreateWithFlags(&c->aux[j], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ev_join[j], cudaEventDisableTiming) == cudaSuccess;
    if (!aux_ok) {
        cudaGetLastError();
        apm_destroy(c);
        return APM_E_CUDA;
    }
    if (fault_alloc() || cudaMalloc((void**)&c->d_status, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        apm_destroy(c);
        return fault_alloc() ? APM_E_NOMEM : APM_E_CUDA;
    }
    if (cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess || fft_configure() != cudaSuccess) {
        cudaGetLastError();
        apm_destroy(c);
        return APM_E_CUDA;
    }
    *out = c;
    return APM_OK;
}

void apm_destroy(apm_ctx* c) {
    if (!c) return;
    free_hierarchy(c);
    profile_free(c->prof);
    for (int j = 0; j < apm_ctx::kAux; ++j) {
        if (c->aux[j]) cudaStreamDestroy(c->aux[j]);
        if (c->ev_join[j]) cudaEventDestroy(c->ev_join[j]);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->d_status) cudaFree(c->d_status);
    delete c;
}

apm_status apm_validate_hierarchy(const apm_config* cfg, const apm_grid* grids, int32_t n) {
    if (!cfg || !grids || cfg->refine != 2 || !(cfg->pad_factor >= 0) || !(cfg->a_over_dx > 0))
        return APM_E_INVALID;
    return validate(*cfg, grids, n);
}

int32_t apm_num_levels(const apm_ctx* c) { return (c && c->has_hier) ? (int32_t)c->levels.size() : 0; }

apm_status apm_get_grid_info(const apm_ctx* c, int32_t grid, apm_grid_info* out) {
    if (!c || !out) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (grid < 0 || grid >= (int)c->grids.size()) return APM_E_INVALID;
    const Level& L = c->levels[c->level_of[grid]];
    const GridDev& g = L.hg[c->index_in_level[grid]];
    out->level = L.level;
    out->border = (g.G[0] - g.N[0]) / 2;
    for (int j = 0; j < 3; ++j) {
        out->gmf[j] = g.G[j];
        out->fft[j] = g.M[j];
        out->phi_short[j] = g.W[j];
        out->field[j] = g.N[j] + 2;
    }
    out->level_index = c->index_in_level[grid];
    out->delta = g.delta;
    out->phi_short_comps = c->cfg.gradient == APM_GRAD_SPECTRAL ? 4 : 1;
    return APM_OK;
}

apm_status apm_set_hierarchy(apm_ctx* c, const apm_grid* grids, int32_t n) {
    Range nvtx_range("apm_set_hierarchy");
    if (!c || !grids) return APM_E_INVALID;
    apm_status st = validate(c->cfg, grids, n);
    if (st != APM_OK) return st;
    // fixed-point positions: 2^-31 root cells, at least 11 fraction bits on the
    // finest level, |x / delta0| 2^31 < 2^51
    {
        int maxlev = 0;
        for (int i = 0; i < n; ++i) maxlev = std::max(maxlev, grids[i].level);
        if (maxlev > 20 || grids[0].dims[0] > (1 << 20)) return APM_E_UNSUPPORTED;
    }
    if (c->has_hier) free_hierarchy(c);
    const apm_config& cfg = c->cfg;
    const bool periodic = cfg.root_bc == APM_BC_PERIODIC;
    const bool f64 = cfg.precision == APM_FP64;
    const size_t csz = f64 ? sizeof(double2) : sizeof(float2);
    const int B = border_cells(cfg);
    const int N0 = grids[0].dims[0];
    c->grids.assign(grids, grids + n);
    int nlev = 0;
    for (int i = 0; i < n; ++i) nlev = std::max(nlev, grids[i].level + 1);
    c->levels.assign(nlev, Level());
    c->level_of.assign(n, 0);
    c->index_in_level.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        Level& L = c->levels[grids[i].level];
        L.level = grids[i].level;
        c->level_of[i] = grids[i].level;
        c->index_in_level[i] = (int)L.grids.size();
        L.grids.push_back(i);
    }
    // ---- per-grid plans
    std::map<int, int> tw_off;       // L -> offset
    int tw_total = 0;
    using TabKey = std::tuple<int, int, int, int, double, double, double>;
    std::map<TabKey, long long> tab_off;
    std::vector<std::pair<TabKey, long long>> tab_list;
    long long tab_total = 0, tab_max = 0;
    auto twiddle = [&](int L) {
        auto it = tw_off.find(L);
        if (it != tw_off.end()) return it->second;
        int o = tw_total;
        tw_off[L] = o;
        tw_total += L;
        return o;
    };
    size_t wsA_max = 0, wsB_max = 0;
    for (Level& L : c->levels) {
        L.max_radix = f64 ? 8 : fft_max_radix();
        long long offA = 0, offB = 0;
        for (int gi : L.grids) {
            const apm_grid& a = grids[gi];
            GridDev g;
            std::memset(&g, 0, sizeof(g));
            const double delta = cfg.box / ((double)N0 * std::pow((double)cfg.refine, a.level));
            const double a_lev = cfg.a_over_dx * delta;
            g.delta = delta;
            g.grad = cfg.gradient;
            g.h = cfg.gradient == APM_GRAD_FD4 ? 3 : 2;
            for (int j = 0; j < 3; ++j) {
                g.N[j] = a.dims[j];
                g.start[j] = a.start[j];
                g.W[j] = a.dims[j] + 2 * g.h;
            }
            double a_par = 0.0;
            if (a.level == 0) {
                g.kind = periodic ? 1 : 2;
                g.mode = periodic ? 2 : 1;
                for (int j = 0; j < 3; ++j) {
                    g.G[j] = a.dims[j];
                    g.M[j] = periodic ? a.dims[j]
                                      : (cfg.gradient == APM_GRAD_FD4 ? even_smooth7_at_least(2 * a.dims[j] + 2)
                                                                      : 2 * a.dims[j]);
                    g.lo[j] = 0;
                    g.s0[j] = ((g.M[j] - g.h) % g.M[j] + g.M[j]) % g.M[j];
                }
                g.parent = -1;
            } else {
                g.kind = 0;
                g.mode = 0;
                a_par = cfg.refine * a_lev;
                for (int j = 0; j < 3; ++j) {
                    g.G[j] = a.dims[j] + 2 * B;
                    g.M[j] = smooth7_at_least(a.dims[j] + 4 * B);
                    g.lo[j] = a.start[j] - B;
                    g.s0[j] = ((B - g.h) % g.M[j] + g.M[j]) % g.M[j];
                }
                const apm_grid& p = grids[a.parent];
                g.parent = c->index_in_level[a.parent];
                for (int j = 0; j < 3; ++j) {
                    g.pN[j] = p.dims[j];
                    g.pstart[j] = p.start[j];
                }
            }
            for (int j = 0; j < 3; ++j) {
                if (g.M[j] > kMaxFft || g.M[j] < 2) return APM_E_UNSUPPORTED;
            }
            // 32-bit cell indices inside the kernels
            if ((long long)g.G[0] * g.G[1] * g.G[2] >= (1LL << 31) ||
                (long long)g.W[0] * g.W[1] * g.W[2] * (cfg.gradient == APM_GRAD_SPECTRAL ? 4 : 1) >= (1LL << 31))
                return APM_E_UNSUPPORTED;
            FftPlan1D* pls[3] = {&g.fx, &g.fy, &g.fz};
            for (int j = 0; j < 3; ++j) {
                if (!fft_plan(g.M[j], f64 ? 8 : L.max_radix, pls[j])) return APM_E_UNSUPPORTED;
                pls[j]->tw_off = twiddle(g.M[j]);
            }
            fft_plan_reversed(g.fy, &g.iy);
            fft_plan_reversed(g.fz, &g.iz);
            g.Hx = g.M[0] / 2 + 1;
            g.Hy2 = g.M[1] / 2 + 1;
            g.Hz2 = g.M[2] / 2 + 1;
            g.cells_gmf = (long long)g.G[0] * g.G[1] * g.G[2];
            g.inv2d = 0.5 / delta;
            g.inv12d = 1.0 / (12.0 * delta);
            for (int j = 0; j < 3; ++j) g.dk[j] = 2.0 * kPiHost / ((double)g.M[j] * delta);
            g.inv_m3 = 1.0 / ((double)g.M[0] * (double)g.M[1] * (double)g.M[2]);
            g.rows_gas = std::max(1, kChunkCells / g.G[0]);
            // 2x2x2 output blocks pair level cells (2k+1, 2k+2), the two children
            // between the same parent centres
            for (int j = 0; j < 3; ++j) {
                const long long ic0 = g.start[j] - 1;       // output cell 0 (cell -1)
                g.acc_sh[j] = (ic0 & 1) ? 0 : 1;
                g.acc_nb[j] = (g.N[j] + 2 + g.acc_sh[j] + 1) / 2;
            }
            // green table (cached per shape and level parameters)
            TabKey key{g.kind, g.M[0], g.M[1], g.M[2], delta, a_lev, a_par};
            auto it = tab_off.find(key);
            if (it == tab_off.end()) {
                long long sz = (long long)g.Hx * g.Hy2 * g.Hz2;
                tab_off[key] = tab_total;
                tab_list.push_back({key, tab_total});
                g.tab_off = tab_total;
                tab_total += sz;
                tab_max = std::max(tab_max, sz);
            } else {
                g.tab_off = it->second;
            }
            // workspace
            const long long Hx = g.Hx;
            long long szA = std::max((long long)g.G[1] * g.G[2], (long long)g.W[2] * g.M[1]) * Hx;
            long long szB = std::max((long long)g.G[2] * g.M[1], (long long)g.W[2] * g.W[1]) * Hx;
            g.wsA = offA;
            g.wsB = offB;
            offA += (szA + 31) / 32 * 32;
            offB += (szB + 31) / 32 * 32;
            L.hg.push_back(g);
        }
        wsA_max = std::max(wsA_max, (size_t)offA);
        wsB_max = std::max(wsB_max, (size_t)offB);
    }
    // ---- device arenas
    if ((st = dmalloc(c, (void**)&c->tw64, tw_total * sizeof(double2))) != APM_OK) return st;
    if ((st = dmalloc(c, (void**)&c->tw32, tw_total * sizeof(float2))) != APM_OK) return st;
    if ((st = dmalloc(c, (void**)&c->tab64, tab_total * sizeof(double))) != APM_OK) return st;
    if (!f64 && (st = dmalloc(c, (void**)&c->tab32, tab_total * sizeof(float))) != APM_OK) return st;
    if ((st = dmalloc(c, &c->wsA, wsA_max * csz)) != APM_OK) return st;
    if ((st = dmalloc(c, &c->wsB, wsB_max * csz)) != APM_OK) return st;
    if (cfg.gradient == APM_GRAD_SPECTRAL && (st = dmalloc(c, &c->wsC, wsB_max * csz)) != APM_OK) return st;
    double* scratch = nullptr;
    if ((st = dmalloc(c, (void**)&scratch, tab_max * sizeof(double))) != APM_OK) return st;
    for (auto& kv : tw_off)
        if (launch_twiddles(c->tw64 + kv.second, c->tw32 + kv.second, kv.first, 0) != cudaSuccess)
            return APM_E_CUDA;
    for (auto& t : tab_list) {
        const TabKey& k = t.first;
        int M[3] = {std::get<1>(k), std::get<2>(k), std::get<3>(k)};
        if (launch_green_table(std::get<0>(k), M, std::get<4>(k), std::get<5>(k), std::get<6>(k),
                               cfg.root_correction, cfg.gradient, c->tab64 + t.second, scratch, 0) != cudaSuccess)
            return APM_E_CUDA;
    }
    if (!f64 && launch_to_f32(c->tab64, c->tab32, tab_total, 0) != cudaSuccess) return APM_E_CUDA;
    // ---- per-level device data
    for (Level& L : c->levels) {
        const int ng = (int)L.grids.size();
        if ((st = upload(c, &L.d_grids, L.hg)) != APM_OK) return st;
        std::vector<Chunk> gas, acc;
        L.acc_first.assign(ng + 1, 0);
        for (int k = 0; k < ng; ++k) {
            L.acc_first[k] = (int)acc.size();
            const GridDev& g = L.hg[k];
            const long long grows = (long long)g.G[1] * g.G[2];
            for (long long t = 0; t < (grows + g.rows_gas - 1) / g.rows_gas; ++t) gas.push_back({k, (int)t});
            const long long nblocks = (long long)g.acc_nb[0] * g.acc_nb[1] * g.acc_nb[2];
            for (long long t = 0; t < (nblocks + kAccBlocksPerCta - 1) / kAccBlocksPerCta; ++t)
                acc.push_back({k, (int)t});
        }
        L.acc_first[ng] = (int)acc.size();
        for (int q = 0; q < kFftPasses; ++q) {
            if ((st = build_pass(c, L, q, f64 ? kFftBudgetF64 : kFftBudgetF32, kFftThreads, f64, L.pass[q])) != APM_OK)
                return st;
            apply_pass(L, q);
        }
        if (cudaMemcpy(L.d_grids, L.hg.data(), L.hg.size() * sizeof(GridDev), cudaMemcpyHostToDevice) != cudaSuccess)
            return APM_E_CUDA;
        if ((st = upload(c, &L.d_gas, gas)) != APM_OK) return st;
        if ((st = upload(c, &L.d_acc, acc)) != APM_OK) return st;
        L.n_gas = (int)gas.size(); L.n_acc = (int)acc.size();
        // tile map
        LevelDev& D = L.dev;
        std::memset(&D, 0, sizeof(D));
        D.level = L.level;
        D.n = ng;
        D.is_root = L.level == 0;
        D.refine = cfg.refine;
        D.g = L.d_grids;
        D.delta = L.hg[0].delta;
        D.inv_delta = 1.0 / D.delta;
        D.delta0 = cfg.box / N0;
        D.inv_delta0 = 1.0 / D.delta0;
        {
            int ex = 0;
            // delta0 = 2^(ex-1): X = rint(x 2^pos_exp) from the bits of x (the
            // exponent bound keeps subnormal coordinates below half a unit)
            const bool pow2 = std::frexp(D.delta0, &ex) == 0.5;
            D.pos_exp = kPosBits - (ex - 1);
            D.delta0_pow2 = (pow2 && D.pos_exp < 1000) ? 1 : 0;
        }
        D.frac_bits = kPosBits - L.level;
        D.span = (long long)N0 << kPosBits;
        D.box = cfg.box;
        D.periodic = periodic ? 1 : 0;
        D.status = c->d_status;
        if (L.level > 0) {
            std::vector<std::pair<std::array<long long, 3>, std::array<long long, 3>>> dep, own;
            long long lo[3] = {1LL << 62, 1LL << 62, 1LL << 62}, hi[3] = {-(1LL << 62), -(1LL << 62), -(1LL << 62)};
            for (const GridDev& g : L.hg) {
                std::array<long long, 3> a, b, ia, ib;
                for (int j = 0; j < 3; ++j) {
                    a[j] = g.lo[j] - 1;
                    b[j] = g.lo[j] + g.G[j] + 1;
                    ia[j] = g.start[j];
                    ib[j] = g.start[j] + g.N[j];
                    lo[j] = std::min(lo[j], a[j]);
                    hi[j] = std::max(hi[j], b[j]);
                }
                dep.push_back({a, b});
                own.push_back({ia, ib});
            }
            long long ext = 0;
            for (int j = 0; j < 3; ++j) ext = std::max(ext, hi[j] - lo[j]);
            int shift = 2;   // tiles of at least 4 cells
            while ((ext >> shift) > 64) ++shift;
            int nt[3];
            for (int j = 0; j < 3; ++j) nt[j] = (int)(((hi[j] - lo[j]) + (1LL << shift) - 1) >> shift);
            std::vector<int> doff, dlist, ooff, olist;
            build_csr(dep, lo, shift, nt, doff, dlist);
            build_csr(own, lo, shift, nt, ooff, olist);
            // dilated occupancy: a particle whose FP32-estimated tile has no
            // occupied neighbour cannot touch any GMF box of the level
            std::vector<unsigned char> occ((size_t)nt[0] * nt[1] * nt[2], 0);
            for (int z = 0; z < nt[2]; ++z)
                for (int y = 0; y < nt[1]; ++y)
                    for (int x = 0; x < nt[0]; ++x) {
                        long long t = x + (long long)nt[0] * (y + (long long)nt[1] * z);
                        if (doff[t + 1] == doff[t]) continue;
                        for (int dz = -1; dz <= 1; ++dz)
                            for (int dy = -1; dy <= 1; ++dy)
                                for (int dx = -1; dx <= 1; ++dx) {
                                    int X = x + dx, Y = y + dy, Z = z + dz;
                                    if (X < 0 || Y < 0 || Z < 0 || X >= nt[0] || Y >= nt[1] || Z >= nt[2]) continue;
                                    occ[X + (size_t)nt[0] * (Y + (size_t)nt[1] * Z)] = 1;
                                }
                    }
            unsigned char* d_occ;
            if ((st = upload(c, &d_occ, occ)) != APM_OK) return st;
            D.map.occ = d_occ;
            int *d_doff, *d_dlist, *d_ooff, *d_olist;
            if ((st = upload(c, &d_doff, doff)) != APM_OK) return st;
            if ((st = upload(c, &d_dlist, dlist)) != APM_OK) return st;
            if ((st = upload(c, &d_ooff, ooff)) != APM_OK) return st;
            if ((st = upload(c, &d_olist, olist)) != APM_OK) return st;
            for (int j = 0; j < 3; ++j) {
                D.map.lo[j] = lo[j];
                D.map.nt[j] = nt[j];
            }
            D.map.shift = shift;
            D.map.dep_off = d_doff; D.map.dep_list = d_dlist;
            D.map.own_off = d_ooff; D.map.own_list = d_olist;
        }
        // pointer tables
        int cap = ng;
        if (L.level > 0) cap = std::max(cap, (int)c->levels[L.level - 1].grids.size());
        L.cap = cap;
        if ((st = dmalloc(c, (void**)&L.d_ptr, (size_t)kRoles * cap * sizeof(void*))) != APM_OK) return st;
        if (cudaMallocHost((void**)&L.h_ptr, (size_t)kRoles * cap * sizeof(void*)) != cudaSuccess) {
            L.h_ptr = nullptr;
            cudaGetLastError();
            return APM_E_NOMEM;
        }
        if (cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) != cudaSuccess) return APM_E_CUDA;
    }
    {
        const int nl = (int)c->levels.size();
        std::vector<LevelDev> lv(nl);
        std::vector<void*> tabs((size_t)kRoles * nl);
        for (int l = 0; l < nl; ++l) {
            lv[l] = c->levels[l].dev;
            for (int r = 0; r < kRoles; ++r)
                tabs[(size_t)r * nl + l] = c->levels[l].d_ptr + (size_t)r * c->levels[l].cap;
        }
        if ((st = upload(c, &c->d_levels, lv)) != APM_OK) return st;
        if ((st = upload(c, &c->d_tabs, tabs)) != APM_OK) return st;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return APM_E_CUDA;
    c->has_hier = true;
    return APM_OK;
}

apm_status apm_deposit(apm_ctx* c, int32_t level, const apm_particles* particles, double half_dt,
                       const double* const* gas, const double* const* parent_gas,
                       int64_t* const* gmf, void* stream) {
    Range nvtx_range("apm_deposit");
    if (!c) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (level < 0 || level >= (int)c->levels.size() || !gmf || !particles_ok(particles))
        return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Level& L = c->levels[level];
    const int ng = (int)L.grids.size();
    for (int i = 0; i < ng; ++i)
        if (!gmf[i]) return APM_E_INVALID;
    void **d_gmf, **d_gas, **d_pgas;
    apm_status st;
    if ((st = set_ptrs(c, L, R_GMF, (const void* const*)gmf, ng, &d_gmf, s)) != APM_OK) return st;
    if ((st = set_ptrs(c, L, R_GAS, (const void* const*)gas, ng, &d_gas, s)) != APM_OK) return st;
    const GridDev* pgrids = nullptr;
    if (level > 0 && parent_gas) {
        Level& P = c->levels[level - 1];
        if ((st = set_ptrs(c, L, R_PGAS, (const void* const*)parent_gas, (int)P.grids.size(), &d_pgas, s)) != APM_OK)
            return st;
        pgrids = P.d_grids;
    } else {
        d_pgas = nullptr;
    }
    {
    Trace t(c, K_GAS, s);
    if (launch_gas_init(L.dev, pgrids, (const double* const*)d_gas, (const double* const*)d_pgas,
                        (int64_t* const*)d_gmf, L.d_gas, L.n_gas, c->cfg.mass_frac_bits,
                        s) != cudaSuccess)
        return APM_E_CUDA;
    }
    Particles P = to_dev(particles);
    if (c->dep_tiles) use_order(c, P);
    Trace t(c, K_DEPOSIT, s);
    return cuda_status(launch_deposit(L.dev, P, half_dt, c->cfg.box, c->cfg.mass_frac_bits,
                                      (int64_t* const*)d_gmf, c->d_status, s));
}

apm_status apm_deposit_all(apm_ctx* c, const apm_particles* particles, double half_dt,
                           const double* const* gas, int64_t* const* gmf, void* stream) {
    Range nvtx_range("apm_deposit_all");
    if (!c) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (!gmf || !particles_ok(particles)) return APM_E_INVALID;
    const int n = (int)c->grids.size(), nl = (int)c->levels.size();
    for (int i = 0; i < n; ++i)
        if (!gmf[i]) return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    apm_status st;
    // baryons of every level (the parent's gas borders each child), as apm_deposit
    std::vector<const void*> pg, pgas, pgm;
    for (int l = 0; l < nl; ++l) {
        Level& L = c->levels[l];
        const int ng = (int)L.grids.size();
        pg.assign(ng, nullptr);
        for (int k = 0; k < ng; ++k) pg[k] = gmf[L.grids[k]];
        void **d_gmf, **d_gas = nullptr, **d_pgas = nullptr;
        if ((st = set_ptrs(c, L, R_GMF, pg.data(), ng, &d_gmf, s)) != APM_OK) return st;
        const GridDev* pgrids = nullptr;
        if (gas) {
            pgas.assign(ng, nullptr);
            for (int k = 0; k < ng; ++k) pgas[k] = gas[L.grids[k]];
            if ((st = set_ptrs(c, L, R_GAS, pgas.data(), ng, &d_gas, s)) != APM_OK) return st;
            if (l > 0) {
                Level& P = c->levels[l - 1];
                pgm.assign(P.grids.size(), nullptr);
                for (size_t k = 0; k < P.grids.size(); ++k) pgm[k] = gas[P.grids[k]];
                if ((st = set_ptrs(c, L, R_PGAS, pgm.data(), (int)P.grids.size(), &d_pgas, s)) != APM_OK)
                    return st;
                pgrids = P.d_grids;
            }
        }
        Trace t(c, K_GAS, s);
        if (launch_gas_init(L.dev, pgrids, (const double* const*)d_gas, (const double* const*)d_pgas,
                            (int64_t* const*)d_gmf, L.d_gas, L.n_gas, c->cfg.mass_frac_bits,
                            s) != cudaSuccess)
            return APM_E_CUDA;
    }
    Particles P = to_dev(particles);
    if (c->dep_tiles) use_order(c, P);
    Trace t(c, K_DEPOSIT, s);
    return cuda_status(launch_deposit_levels(c->d_levels, nl, P, half_dt, c->cfg.box, c->cfg.mass_frac_bits,
                                             (int64_t* const* const*)(c->d_tabs + (size_t)R_GMF * nl),
                                             c->d_status, s));
}

apm_status apm_solve_level(apm_ctx* c, int32_t level, const int64_t* const* gmf,
                           void* const* phi_short, void* stream) {
    Range nvtx_range("apm_solve_level");
    if (!c) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (level < 0 || level >= (int)c->levels.size() || !gmf || !phi_short) return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Level& L = c->levels[level];
    const int ng = (int)L.grids.size();
    for (int i = 0; i < ng; ++i)
        if (!gmf[i] || !phi_short[i]) return APM_E_INVALID;
    void **d_gmf, **d_phis;
    apm_status st;
    if ((st = set_ptrs(c, L, R_GMF_IN, (const void* const*)gmf, ng, &d_gmf, s)) != APM_OK) return st;
    if ((st = set_ptrs(c, L, R_PHIS, (const void* const*)phi_short, ng, &d_phis, s)) != APM_OK) return st;
    const Kern kind[kFftPasses] = {K_XF, K_YF, K_Z, K_YI, K_XI};
    const int ncomp = c->cfg.gradient == APM_GRAD_SPECTRAL ? 4 : 1;
    // batched: each pass is one launch over every grid of the level; otherwise
    // one launch sequence per grid, grid after grid
    const int g_first = c->batched ? -1 : 0, g_last = c->batched ? -1 : ng - 1;
    for (int gk = g_first; gk <= g_last; ++gk) {
        for (int q = 0; q < kFftPasses; ++q) {
            // a y pass fused into its x pass launches nothing (and is not traced)
            const PassPlan& P = L.pass[q];
            if (gk < 0 ? P.seg.empty() : P.count[gk] == 0) continue;
            Trace t(c, kind[q], s);
            t.launches(gk < 0 ? (int)P.seg.size() : 1);
            if (run_pass(c, L, q, P, d_gmf, d_phis, s, 0, gk) != cudaSuccess) return APM_E_CUDA;
        }
        // the spectral gradient's acceleration components: z (table times
        // -i D_comp), y inverse and x inverse again on the kept forward transform
        for (int comp = 1; comp < ncomp; ++comp)
            for (int q = kPassZ; q < kFftPasses; ++q) {
                if (gk < 0 ? L.pass[q].seg.empty() : L.pass[q].count[gk] == 0) continue;
                Trace t(c, kind[q], s);
                t.launches(gk < 0 ? (int)L.pass[q].seg.size() : 1);
                if (run_pass(c, L, q, L.pass[q], d_gmf, d_phis, s, comp, gk) != cudaSuccess) return APM_E_CUDA;
            }
    }
    return APM_OK;
}

apm_status apm_set_deposit_tiles(apm_ctx* c, int32_t on) {
    if (!c || (on != 0 && on != 1)) return APM_E_INVALID;
    c->dep_tiles = on == 1;
    return APM_OK;
}

apm_status apm_set_grid_batching(apm_ctx* c, int32_t batched) {
    if (!c || (batched != 0 && batched != 1)) return APM_E_INVALID;
    c->batched = batched == 1;
    return APM_OK;
}

apm_status apm_graph_begin(apm_ctx* c, void* stream) {
    if (!c || !stream) return APM_E_INVALID;   // the legacy default stream cannot be captured
    if (!c->has_hier) return APM_E_STATE;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) return APM_E_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return APM_E_STATE;
    return cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess
               ? APM_OK : APM_E_CUDA;
}

apm_status apm_graph_end(apm_ctx* c, void* stream, int32_t* graph_id) {
    if (!c || !stream || !graph_id) return APM_E_INVALID;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture((cudaStream_t)stream, &g) != cudaSuccess || !g) {
        cudaGetLastError();
        return APM_E_STATE;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return APM_E_CUDA;
    }
    c->graphs.push_back(exec);
    *graph_id = (int32_t)c->graphs.size() - 1;
    return APM_OK;
}

apm_status apm_graph_launch(apm_ctx* c, int32_t graph_id, void* stream) {
    if (!c || graph_id < 0 || graph_id >= (int32_t)c->graphs.size() || !c->graphs[graph_id]) return APM_E_INVALID;
    return cudaGraphLaunch(c->graphs[graph_id], (cudaStream_t)stream) == cudaSuccess ? APM_OK : APM_E_CUDA;
}

apm_status apm_graph_destroy(apm_ctx* c, int32_t graph_id) {
    if (!c || graph_id < 0 || graph_id >= (int32_t)c->graphs.size() || !c->graphs[graph_id]) return APM_E_INVALID;
    cudaGraphExecDestroy(c->graphs[graph_id]);
    c->graphs[graph_id] = nullptr;
    return APM_OK;
}

apm_status apm_reserve_order(apm_ctx* c, int64_t n_max) {
    Range nvtx_range("apm_reserve_order");
    if (!c || n_max < 0 || n_max > (int64_t)INT32_MAX) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    apm_ctx::Order& o = c->order;
    if (cudaDeviceSynchronize() != cudaSuccess) return APM_E_CUDA;
    for (void* p : {(void*)o.count, (void*)o.sums, (void*)o.key, (void*)o.rank, (void*)o.perm})
        if (p) dfree(c, p);
    o = apm_ctx::Order();
    if (n_max == 0) return APM_OK;
    // bins of 2^shift root cells, at least 4 per side, at most 128^3 bins (so
    // the scan's chunk totals fit one CTA)
    const int N0 = c->grids[0].dims[0];
    int shift = 2;
    while (((N0 + (1 << shift) - 1) >> shift) > 128) ++shift;
    const int nb = (N0 + (1 << shift) - 1) >> shift;
    const size_t nbins = (size_t)nb * nb * nb;
    apm_status st;
    if ((st = dmalloc(c, (void**)&o.count, nbins * sizeof(unsigned))) != APM_OK ||
        (st = dmalloc(c, (void**)&o.sums, 1024 * sizeof(unsigned))) != APM_OK ||
        (st = dmalloc(c, (void**)&o.key, (size_t)n_max * sizeof(unsigned))) != APM_OK ||
        (st = dmalloc(c, (void**)&o.rank, (size_t)n_max * sizeof(unsigned))) != APM_OK ||
        (st = dmalloc(c, (void**)&o.perm, (size_t)n_max * sizeof(int))) != APM_OK) {
        for (void* p : {(void*)o.count, (void*)o.sums, (void*)o.key, (void*)o.rank, (void*)o.perm})
            if (p) dfree(c, p);
        o = apm_ctx::Order();
        return st;
    }
    o.cap = n_max;
    o.shift = shift;
    o.nb = nb;
    return APM_OK;
}

apm_status apm_order_particles(apm_ctx* c, const apm_particles* particles, double half_dt, void* stream) {
    Range nvtx_range("apm_order_particles");
    if (!c || !particles_ok(particles)) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    apm_ctx::Order& o = c->order;
    if (!o.perm || particles->n > o.cap) return APM_E_INVALID;
    Particles P = to_dev(particles);
    Trace t(c, K_ORDER, (cudaStream_t)stream);
    if (launch_order(c->levels[0].dev, P, half_dt, o.shift, o.nb, o.count, o.sums, o.key, o.rank, o.perm,
                     (cudaStream_t)stream) != cudaSuccess)
        return APM_E_CUDA;
    o.n = P.n;
    return APM_OK;
}

apm_status apm_autotune_level(apm_ctx* c, int32_t level, const int64_t* const* gmf,
                              void* const* phi_short, void* stream) {
    Range nvtx_range("apm_autotune_level");
    if (!c) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (level < 0 || level >= (int)c->levels.size() || !gmf || !phi_short) return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return APM_E_STATE;
    Level& L = c->levels[level];
    const int ng = (int)L.grids.size();
    for (int i = 0; i < ng; ++i)
        if (!gmf[i] || !phi_short[i]) return APM_E_INVALID;
    void **d_gmf, **d_phis;
    apm_status st;
    if ((st = set_ptrs(c, L, R_GMF_IN, (const void* const*)gmf, ng, &d_gmf, s)) != APM_OK) return st;
    if ((st = set_ptrs(c, L, R_PHIS, (const void* const*)phi_short, ng, &d_phis, s)) != APM_OK) return st;
    const bool f64 = c->cfg.precision == APM_FP64;
    const std::vector<int> budgets = f64 ? std::vector<int>{256, 512, 1024, 2048, 4096}
                                         : std::vector<int>{512, 1024, 2048, 4096, 8192};
    const int threads[] = {128, 256};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return APM_E_CUDA;
    }
    auto upload_grids = [&]() -> apm_status {
        if (cudaStreamSynchronize(s) != cudaSuccess ||
            cudaMemcpy(L.d_grids, L.hg.data(), L.hg.size() * sizeof(GridDev), cudaMemcpyHostToDevice) != cudaSuccess)
            return APM_E_CUDA;
        return APM_OK;
    };
    // the fastest of kTuneLaunches timed launches after a warm one (the
    // minimum: launch-to-launch noise only adds time).  The passes are tuned
    // in order, so each candidate reads the previous pass's output and
    // rewrites the same result (the shape never changes a value).
    constexpr int kTuneLaunches = 5;
    auto time_pass = [&](int q, const PassPlan& P, float* ms) -> apm_status {
        for (size_t k = 0; k < L.hg.size(); ++k) L.hg[k].lines[q] = P.lines[k];
        apm_status r = upload_grids();
        if (r != APM_OK) return r;
        if (run_pass(c, L, q, P, d_gmf, d_phis, s) != cudaSuccess) return APM_E_CUDA;
        float best = 0;
        for (int k = 0; k < kTuneLaunches; ++k) {
            float t = 0;
            if (cudaEventRecord(e0, s) != cudaSuccess ||
                run_pass(c, L, q, P, d_gmf, d_phis, s) != cudaSuccess ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                return APM_E_CUDA;
            best = k == 0 ? t : std::min(best, t);
        }
        *ms = best;
        return APM_OK;
    };
    // the launch shapes are those of the runtime-planned kernels: tune them with
    // every pass on that kernel, then choose each pass's plan below
    const int plan0[kFftPasses] = {L.plan[0], L.plan[1], L.plan[2], L.plan[3], L.plan[4]};
    if (!f64) {
        for (int q = 0; q < kFftPasses; ++q) L.plan[q] = 1;
        for (int q = 0; q < kFftPasses && st == APM_OK; ++q) {
            PassPlan P;
            if ((st = build_pass(c, L, q, L.pass[q].budget, L.pass[q].threads, f64, P)) != APM_OK) break;
            dfree(c, L.pass[q].d);
            L.pass[q] = P;
            apply_pass(L, q);
        }
        if (st == APM_OK) st = upload_grids();
    }
    for (int q = 0; q < kFftPasses && st == APM_OK; ++q) {
        float best_ms = 0;
        st = time_pass(q, L.pass[q], &best_ms);
        for (size_t bi = 0; bi < budgets.size() && st == APM_OK; ++bi) {
            for (int t : threads) {
                PassPlan cand;
                if ((st = build_pass(c, L, q, budgets[bi], t, f64, cand)) != APM_OK) break;
                float ms = 0;
                const bool same = cand.lines == L.pass[q].lines && cand.threads == L.pass[q].threads;
                if (!same && (st = time_pass(q, cand, &ms)) == APM_OK && ms < best_ms) {
                    best_ms = ms;
                    dfree(c, L.pass[q].d);
                    L.pass[q] = cand;
                } else {
                    dfree(c, cand.d);
                }
                if (st != APM_OK) break;
            }
        }
        apply_pass(L, q);
        if (st == APM_OK) st = upload_grids();
        // the chosen shape leaves this pass's output in place for the next pass
        if (st == APM_OK && run_pass(c, L, q, L.pass[q], d_gmf, d_phis, s) != cudaSuccess) st = APM_E_CUDA;
    }
    // whole-level choices, each timed over the five passes (the fastest of
    // kTuneLaunches level solves after a warm one): the kernel of each pass
    // (compile-time plan or runtime plan, FP32), the grid packing, and the
    // runtime plans' largest radix (FP32).  A different plan or radix rounds
    // differently (both within the FP32 tolerances, tested); the packing only
    // reorders work.
    const int ncomp_t = c->cfg.gradient == APM_GRAD_SPECTRAL ? 4 : 1;
    auto rebuild = [&]() -> apm_status {
        for (int q = 0; q < kFftPasses; ++q) {
            PassPlan P;
            apm_status r = build_pass(c, L, q, L.pass[q].budget, L.pass[q].threads, f64, P);
            if (r != APM_OK) return r;
            dfree(c, L.pass[q].d);
            L.pass[q] = P;
            apply_pass(L, q);
        }
        return upload_grids();
    };
    auto time_level = [&](float* ms) -> apm_status {
        float best = 0;
        for (int k = 0; k <= kTuneLaunches; ++k) {
            float t = 0;
            if (cudaEventRecord(e0, s) != cudaSuccess) return APM_E_CUDA;
            for (int q = 0; q < kFftPasses; ++q)
                if (run_pass(c, L, q, L.pass[q], d_gmf, d_phis, s) != cudaSuccess) return APM_E_CUDA;
            for (int comp = 1; comp < ncomp_t; ++comp)
                for (int q = kPassZ; q < kFftPasses; ++q)
                    if (run_pass(c, L, q, L.pass[q], d_gmf, d_phis, s, comp) != cudaSuccess) return APM_E_CUDA;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                return APM_E_CUDA;
            if (k == 1 || (k > 1 && t < best)) best = t;   // launch 0 warms
        }
        *ms = best;
        return APM_OK;
    };
    // one knob at a time: keep the candidate when it is faster, else restore
    auto try_knob = [&](auto set, auto restore) -> apm_status {
        float base = 0, cand = 0;
        apm_status r = time_level(&base);
        if (r != APM_OK) return r;
        set();
        if ((r = rebuild()) != APM_OK || (r = time_level(&cand)) != APM_OK) return r;
        if (cand < base) return APM_OK;
        restore();
        return rebuild();
    };
    if (st == APM_OK && !f64) {
        // each pass: the compile-time plan (where its lengths have one) against
        // the tuned runtime-planned kernel
        for (int q = 0; q < kFftPasses && st == APM_OK; ++q) {
            bool any_fast = false;
            for (int k = 0; k < (int)L.hg.size(); ++k) {
                const GridDev& g = L.hg[k];
                const int len = (q == kPassXf || q == kPassXi) ? g.M[0] : (q == kPassZ ? g.M[2] : g.M[1]);
                any_fast = any_fast || fast_length(len);
            }
            if (any_fast && fft_fast_enabled())
                st = try_knob([&] { L.plan[q] = 0; }, [&] { L.plan[q] = 1; });
            else
                L.plan[q] = plan0[q];
        }
        if (st == APM_OK) st = rebuild();
        // the fused plane kernels: x + y forward, y + x inverse (grids with
        // M0 = M1 whose plane fits)
        bool any_fuse = false;
        for (const GridDev& g : L.hg) any_fuse = any_fuse || (g.M[0] == g.M[1] && fast_xy_length(g.M[0]));
        if (any_fuse && fft_fast_enabled()) {
            for (int q : {(int)kPassXf, (int)kPassXi}) {
                if (st != APM_OK) break;
                const int old = L.plan[q];
                st = try_knob([&] { L.plan[q] = 2; }, [&] { L.plan[q] = old; });
            }
        }
    }
    if (st == APM_OK && L.hg.size() > 1) {
        const int old = L.packing;
        st = try_knob([&] { L.packing = 1 - old; }, [&] { L.packing = old; });
    }
    if (st == APM_OK && !f64) {
        const int old = L.max_radix, alt = old == 16 ? 8 : 16;
        st = try_knob([&] { replan_level(L, alt); }, [&] { replan_level(L, old); });
    }
    // the chosen shapes leave the level's potential in phi_short
    for (int q = 0; q < kFftPasses && st == APM_OK; ++q)
        if (run_pass(c, L, q, L.pass[q], d_gmf, d_phis, s) != cudaSuccess) st = APM_E_CUDA;
    // the spectral gradient's other components with the chosen shapes
    const int ncomp = c->cfg.gradient == APM_GRAD_SPECTRAL ? 4 : 1;
    for (int comp = 1; comp < ncomp && st == APM_OK; ++comp)
        for (int q = kPassZ; q < kFftPasses && st == APM_OK; ++q)
            if (run_pass(c, L, q, L.pass[q], d_gmf, d_phis, s, comp) != cudaSuccess) st = APM_E_CUDA;
    if (st != APM_OK) {   // keep the descriptors consistent with the plans in use
        for (int q = 0; q < kFftPasses; ++q) apply_pass(L, q);
        cudaStreamSynchronize(s);
        cudaMemcpy(L.d_grids, L.hg.data(), L.hg.size() * sizeof(GridDev), cudaMemcpyHostToDevice);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

apm_status apm_get_fft_shapes(const apm_ctx* c, int32_t level, apm_fft_shapes* out) {
    if (!c || !out) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (level < 0 || level >= (int)c->levels.size()) return APM_E_INVALID;
    const Level& L = c->levels[level];
    for (int q = 0; q < kFftPasses; ++q) {
        out->budget[q] = L.pass[q].budget;
        out->threads[q] = L.pass[q].threads;
        out->plan[q] = L.plan[q];
    }
    out->max_radix = L.max_radix;
    out->packing = L.packing;
    return APM_OK;
}

apm_status apm_get_pass_kernels(const apm_ctx* c, int32_t level, int32_t pass, int32_t* kinds, int32_t n) {
    if (!c || !kinds) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (level < 0 || level >= (int)c->levels.size() || pass < 0 || pass >= kFftPasses) return APM_E_INVALID;
    const Level& L = c->levels[level];
    const PassPlan& P = L.pass[pass];
    if (n != (int)L.hg.size() || (int)P.count.size() != n) return APM_E_INVALID;
    for (int k = 0; k < n; ++k) {
        if (P.count[k] == 0) {
            kinds[k] = 3;
            continue;
        }
        const int f = P.seg[P.seg_of[k]].fast_L;
        kinds[k] = f < 0 ? 2 : (f > 0 ? 1 : 0);
    }
    return APM_OK;
}

apm_status apm_set_fft_shapes(apm_ctx* c, int32_t level, const apm_fft_shapes* shapes) {
    if (!c || !shapes) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (level < 0 || level >= (int)c->levels.size()) return APM_E_INVALID;
    const bool f64 = c->cfg.precision == APM_FP64;
    for (int q = 0; q < kFftPasses; ++q) {
        const int t = shapes->threads[q];
        if (shapes->budget[q] < 1 || (t != 128 && t != 256)) return APM_E_INVALID;
        const int pmax = (q == kPassXf || q == kPassXi) ? 2 : 1;   // 2: fused with the y pass
        if (shapes->plan[q] < 0 || shapes->plan[q] > pmax) return APM_E_INVALID;
    }
    if ((shapes->packing != 0 && shapes->packing != 1) ||
        (shapes->max_radix != 8 && shapes->max_radix != 16) || (f64 && shapes->max_radix != 8))
        return APM_E_INVALID;
    Level& L = c->levels[level];
    if (cudaDeviceSynchronize() != cudaSuccess) return APM_E_CUDA;
    for (int q = 0; q < kFftPasses; ++q) L.plan[q] = shapes->plan[q];
    L.packing = shapes->packing;
    if (shapes->max_radix != L.max_radix && !replan_level(L, shapes->max_radix)) return APM_E_UNSUPPORTED;
    for (int q = 0; q < kFftPasses; ++q) {
        PassPlan P;
        apm_status st = build_pass(c, L, q, shapes->budget[q], shapes->threads[q], f64, P);
        if (st != APM_OK) return st;
        dfree(c, L.pass[q].d);
        L.pass[q] = P;
        apply_pass(L, q);
    }
    return cudaMemcpy(L.d_grids, L.hg.data(), L.hg.size() * sizeof(GridDev), cudaMemcpyHostToDevice) == cudaSuccess
               ? APM_OK : APM_E_CUDA;
}

apm_status apm_accel(apm_ctx* c, int32_t level, const void* const* phi_short,
                     const void* const* parent_phi, const void* const* parent_acc, void* const* phi,
                     void* const* acc, void* stream) {
    Range nvtx_range("apm_accel");
    if (!c) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (level < 0 || level >= (int)c->levels.size() || !phi_short || !phi || !acc) return APM_E_INVALID;
    if ((parent_phi == nullptr) != (parent_acc == nullptr)) return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Level& L = c->levels[level];
    const int ng = (int)L.grids.size();
    void **d_phis, **d_pphi = nullptr, **d_pacc = nullptr, **d_phi, **d_acc;
    apm_status st;
    if ((st = set_ptrs(c, L, R_PHIS_IN, phi_short, ng, &d_phis, s)) != APM_OK) return st;
    if ((st = set_ptrs(c, L, R_PHI, (const void* const*)phi, ng, &d_phi, s)) != APM_OK) return st;
    if ((st = set_ptrs(c, L, R_ACC, (const void* const*)acc, ng, &d_acc, s)) != APM_OK) return st;
    const GridDev* pgrids = nullptr;
    if (parent_phi && level > 0) {
        Level& P = c->levels[level - 1];
        int np = (int)P.grids.size();
        if ((st = set_ptrs(c, L, R_PPHI, parent_phi, np, &d_pphi, s)) != APM_OK) return st;
        if ((st = set_ptrs(c, L, R_PACC, parent_acc, np, &d_pacc, s)) != APM_OK) return st;
        pgrids = P.d_grids;
    }
    const int grad = c->cfg.gradient;
    // batched: one launch over every grid; otherwise one launch per grid
    const int g_first = c->batched ? -1 : 0, g_last = c->batched ? -1 : ng - 1;
    for (int gk = g_first; gk <= g_last; ++gk) {
        const Chunk* ch = gk < 0 ? L.d_acc : L.d_acc + L.acc_first[gk];
        const int nch = gk < 0 ? L.n_acc : L.acc_first[gk + 1] - L.acc_first[gk];
        Trace t(c, K_ACCEL, s);
        cudaError_t e;
        if (grad == APM_GRAD_FD2)
            e = c->cfg.precision == APM_FP64
                ? launch_accel<double>(L.dev, pgrids, (const void* const*)d_phis, (const void* const*)d_pphi,
                                       (const void* const*)d_pacc, d_phi, d_acc, ch, nch, s)
                : launch_accel<float>(L.dev, pgrids, (const void* const*)d_phis, (const void* const*)d_pphi,
                                      (const void* const*)d_pacc, d_phi, d_acc, ch, nch, s);
        else
            e = c->cfg.precision == APM_FP64
                ? launch_accel_var<double>(L.dev, pgrids, (const void* const*)d_phis, (const void* const*)d_pphi,
                                             (const void* const*)d_pacc, d_phi, d_acc, ch, nch, grad, s)
                : launch_accel_var<float>(L.dev, pgrids, (const void* const*)d_phis, (const void* const*)d_pphi,
                                            (const void* const*)d_pacc, d_phi, d_acc, ch, nch, grad, s);
        if (e != cudaSuccess) return APM_E_CUDA;
    }
    return APM_OK;
}

apm_status apm_interp(apm_ctx* c, int32_t level, const void* const* acc,
                      const apm_particles* particles, double half_dt, void* acc_out, void* stream) {
    Range nvtx_range("apm_interp");
    if (!c) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (level < 0 || level >= (int)c->levels.size() || !acc || !particles_ok(particles) ||
        (!acc_out && particles->n > 0))
        return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    Level& L = c->levels[level];
    void** d_acc;
    apm_status st;
    if ((st = set_ptrs(c, L, R_ACC_IN, acc, (int)L.grids.size(), &d_acc, s)) != APM_OK) return st;
    const LevelDev* finer = level + 1 < (int)c->levels.size() ? &c->levels[level + 1].dev : nullptr;
    Particles P = to_dev(particles);
    use_order(c, P);
    Trace t(c, K_INTERP, s);
    cudaError_t e = c->cfg.precision == APM_FP64
        ? launch_interp<double>(L.dev, finer, P, half_dt, (const void* const*)d_acc, acc_out, s)
        : launch_interp<float>(L.dev, finer, P, half_dt, (const void* const*)d_acc, acc_out, s);
    return cuda_status(e);
}

apm_status apm_interp_all(apm_ctx* c, const void* const* acc, const apm_particles* particles,
                          double half_dt, void* acc_out, void* stream) {
    Range nvtx_range("apm_interp_all");
    if (!c) return APM_E_INVALID;
    if (!c->has_hier) return APM_E_STATE;
    if (!acc || !particles_ok(particles) || (!acc_out && particles->n > 0)) return APM_E_INVALID;
    const int n = (int)c->grids.size(), nl = (int)c->levels.size();
    for (int i = 0; i < n; ++i)
        if (!acc[i]) return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<const void*> pa;
    for (int l = 0; l < nl; ++l) {
        Level& L = c->levels[l];
        const int ng = (int)L.grids.size();
        pa.assign(ng, nullptr);
        for (int k = 0; k < ng; ++k) pa[k] = acc[L.grids[k]];
        void** d_acc;
        apm_status st = set_ptrs(c, L, R_ACC_IN, pa.data(), ng, &d_acc, s);
        if (st != APM_OK) return st;
    }
    Particles P = to_dev(particles);
    use_order(c, P);
    const void* const* const* tabs = (const void* const* const*)(c->d_tabs + (size_t)R_ACC_IN * nl);
    Trace t(c, K_INTERP, s);
    cudaError_t e = c->cfg.precision == APM_FP64
        ? launch_interp_levels<double>(c->d_levels, nl, P, half_dt, tabs, acc_out, s)
        : launch_interp_levels<float>(c->d_levels, nl, P, half_dt, tabs, acc_out, s);
    return cuda_status(e);
}

apm_status apm_kick_drift(apm_ctx* c, int64_t n, double* x, double* y, double* z, double* vx, double* vy,
                          double* vz, const void* acc, double dt, void* stream) {
    Range nvtx_range("apm_kick_drift");
    if (!c) return APM_E_INVALID;
    if (n < 0 || (n > 0 && (!x || !y || !z || !vx || !vy || !vz || !acc))) return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = c->cfg.precision == APM_FP64
                        ? launch_kick_drift<double>(n, x, y, z, vx, vy, vz, acc, dt, s)
                        : launch_kick_drift<float>(n, x, y, z, vx, vy, vz, acc, dt, s);
    return cuda_status(e);
}

int32_t apm_kernel_count(void) { return K_COUNT; }

const char* apm_kernel_name(int32_t k) { return (k >= 0 && k < K_COUNT) ? kKernelNames[k] : nullptr; }

apm_status apm_profile_enable(apm_ctx* c, int32_t on, int32_t capacity) {
    if (!c) return APM_E_INVALID;
    cudaDeviceSynchronize();
    profile_free(c->prof);
    Profiler& P = c->prof;
    for (int k = 0; k < K_COUNT; ++k) {
        P.launches[k] = 0;
        P.ms[k] = 0.0;
    }
    if (!on) return APM_OK;
    if (capacity < 1) return APM_E_INVALID;
    P.ev.resize(2 * (size_t)capacity);
    P.kind.assign(capacity, 0);
    P.n_launch.assign(capacity, 1);
    for (cudaEvent_t& e : P.ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
            profile_free(P);
            return APM_E_CUDA;
        }
    P.on = true;
    return APM_OK;
}

apm_status apm_profile_read(apm_ctx* c, int32_t kernel, int64_t* launches, double* total_ms) {
    if (!c || kernel < 0 || kernel >= K_COUNT || !launches || !total_ms) return APM_E_INVALID;
    Profiler& P = c->prof;
    if (P.used > 0) {
        if (cudaDeviceSynchronize() != cudaSuccess) return APM_E_CUDA;
        for (int i = 0; i < P.used; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            P.launches[P.kind[i]] += P.n_launch[i];
            P.ms[P.kind[i]] += ms;
        }
        P.used = 0;
    }
    *launches = P.launches[kernel];
    *total_ms = P.ms[kernel];
    return APM_OK;
}

apm_status apm_sync_status(apm_ctx* c, void* stream) {
    Range nvtx_range("apm_sync_status");
    if (!c) return APM_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return APM_E_CUDA;
    unsigned h = 0;
    if (cudaMemcpy(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
        return APM_E_CUDA;
    if (h && cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess) return APM_E_CUDA;
    if (h & kStOverflow) return APM_E_OVERFLOW;
    if (h & kStOutOfBox) return APM_E_OUT_OF_BOX;
    if (h & kStTimeout) return APM_E_TIMEOUT;
    if (h & kStBounds) return APM_E_BOUNDS;
    return APM_OK;
}

}  // extern "C"

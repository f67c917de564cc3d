// apm_internal.cuh -- device descriptors and kernel entry points shared by the
// translation units of libapm (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "apm.h"

namespace apm {

// ---------------------------------------------------------------------------
// compile-time sizes
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 12;      // radix stages of one 1-D transform
constexpr int kFftThreads = 256;    // most threads of an FFT pass CTA (launch bound)
// complex elements one buffer of a pass CTA aims at by default (lines x length)
constexpr int kFftBudgetF32 = 2048;
constexpr int kFftBudgetF64 = 1024;
constexpr int kFftSmemLimit = 200 * 1024;   // dynamic shared memory a pass CTA may take

// the five FFT passes of a level solve
enum { kPassXf = 0, kPassYf = 1, kPassZ = 2, kPassYi = 3, kPassXi = 4, kFftPasses = 5 };

inline int pow2_floor_i(int v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}
// lines per CTA of a pass for a transform of length L and a buffer budget (in
// complex elements): a power of two; row pairs 1..32 for the x passes, kx
// columns 4..32 (FP64 2..32) for the y/z passes (at least 32 contiguous bytes
// of each row a line group reads)
inline int fft_pass_lines(int pass, int L, int budget, bool f64) {
    const int v = pow2_floor_i(std::max(1, budget / L));
    if (pass == kPassXf || pass == kPassXi) return std::min(32, v);
    return std::min(32, std::max(f64 ? 2 : 4, v));
}
// bytes of the x-forward pass's int64 row staging area (2 lines rows of G0
// cells, rounded to 128 bytes) plus its mbarrier
__host__ __device__ inline size_t fft_xf_stage_bytes(int lines, int G0) {
    return ((size_t)2 * lines * G0 * 8 + 127) / 128 * 128 + 128;
}
// dynamic shared memory of a pass CTA: two buffers plus the twiddles (the x
// passes pad each element row to lines + 1); the x-forward pass also stages
// its GMF rows (G0: the GMF row length)
inline size_t fft_pass_smem(int pass, int L, int lines, size_t csz, int G0 = 0) {
    if (pass == kPassXf) return (size_t)(2 * L * (lines + 1) + L) * csz + fft_xf_stage_bytes(lines, G0);
    if (pass == kPassXi) return (size_t)(2 * L * (lines + 1) + L) * csz;
    return (size_t)(2 * L * lines + L) * csz;
}
constexpr int kMaxFft = 1024;       // longest supported transform

// device status bits (latched with atomicOr, read by apm_sync_status)
constexpr unsigned kStOverflow = 1u;
constexpr unsigned kStOutOfBox = 2u;
constexpr unsigned kStTimeout = 4u;
constexpr unsigned kStBounds = 8u;

// Bounds-checked builds (-DAPM_BOUNDS_CHECK): the kernels test each global
// index whose value depends on the data or the hierarchy before using it; an
// index outside [0, n) sets the status word's bounds bit (apm_sync_status:
// APM_E_BOUNDS) and the access is skipped.  Release builds compile the tests
// out.  Nothing here asserts or traps.
#ifdef APM_BOUNDS_CHECK
__device__ __forceinline__ bool in_bounds(long long i, long long n, unsigned* status) {
    if (i >= 0 && i < n) return true;
    if (status) atomicOr(status, kStBounds);
    return false;
}
#define APM_IN_BOUNDS(i, n, status) ::apm::in_bounds((long long)(i), (long long)(n), (status))
#else
#define APM_IN_BOUNDS(i, n, status) true
#endif

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// One mixed-radix 1-D transform of length L (Stockham, radices in order).
struct FftPlan1D {
    int L;
    int nst;
    int tw_off;                       // offset of exp(-2 pi i t/L), t < L, in the twiddle arenas
    unsigned char radix[kMaxStages];
    // per stage: Ns (product of the radices before it), the twiddle stride
    // L / (Ns R), and ceil(2^32 / Ns) for exact division of small integers
    // (n < 2^21) by Ns as __umulhi(n, magic) (Ns = 1: magic 0, q = n)
    unsigned short ns[kMaxStages];
    unsigned short step[kMaxStages];
    unsigned magic[kMaxStages];
};

// Stage radices of a length-L transform: greedily the largest allowed radix
// (at most max_radix) that divides what is left.  Radices above 8 are
// composites of two of 2, 3, 4, 5, 7, 8 run in registers (FP32 path only).
inline bool fft_plan(int L, int max_radix, FftPlan1D* pl) {
    static const int kSimple[] = {8, 7, 5, 4, 3, 2};
    static const int kWithComposite[] = {16, 15, 14, 12, 10, 9, 8, 7, 6, 5, 4, 3, 2};
    pl->L = L;
    pl->nst = 0;
    if (L < 2) return false;
    int n = L;
    while (n > 1) {
        int pick = 0;
        if (max_radix <= 8) {
            for (int r : kSimple)
                if (n % r == 0) { pick = r; break; }
        } else {
            for (int r : kWithComposite)
                if (r <= max_radix && n % r == 0) { pick = r; break; }
        }
        if (!pick || pl->nst >= kMaxStages) return false;
        pl->radix[pl->nst++] = (unsigned char)pick;
        n /= pick;
    }
    int Ns = 1;
    for (int st = 0; st < pl->nst; ++st) {
        pl->ns[st] = (unsigned short)Ns;
        pl->step[st] = (unsigned short)(L / (Ns * pl->radix[st]));
        pl->magic[st] = Ns == 1 ? 0u : (unsigned)((0x100000000ULL + Ns - 1) / Ns);
        Ns *= pl->radix[st];
    }
    return true;
}

// The same transform with the radices in reverse order (the inverse column
// transforms: the z pass's inverse starts with the radix its forward ends on).
inline void fft_plan_reversed(const FftPlan1D& f, FftPlan1D* r) {
    *r = f;
    for (int st = 0; st < f.nst; ++st) r->radix[st] = f.radix[f.nst - 1 - st];
    int Ns = 1;
    for (int st = 0; st < r->nst; ++st) {
        r->ns[st] = (unsigned short)Ns;
        r->step[st] = (unsigned short)(r->L / (Ns * r->radix[st]));
        r->magic[st] = Ns == 1 ? 0u : (unsigned)((0x100000000ULL + Ns - 1) / Ns);
        Ns *= r->radix[st];
    }
}

// ---- FP32 transforms with compile-time plans (fft_fast.cuh) ------------------
// Lengths with a compile-time radix plan: X(L, R1, R2, R3); R3 = 1 for two
// stages.  Every radix is one the FP32 butterflies compute in registers.
#define APM_FAST_LENGTHS(X) \
    X(36, 6, 6, 1) X(40, 8, 5, 1) X(42, 7, 6, 1) X(45, 9, 5, 1) X(48, 8, 6, 1) X(49, 7, 7, 1) \
    X(50, 10, 5, 1) X(54, 9, 6, 1) X(56, 8, 7, 1) X(60, 10, 6, 1) X(63, 9, 7, 1) X(64, 8, 8, 1) \
    X(70, 10, 7, 1) X(72, 9, 8, 1) X(75, 15, 5, 1) X(80, 10, 8, 1) X(81, 9, 9, 1) X(84, 12, 7, 1) \
    X(128, 16, 8, 1) X(150, 15, 10, 1) X(256, 16, 16, 1) X(512, 8, 8, 8)
constexpr int kFastTx = 16;   // kx columns per CTA of a fast column pass
constexpr int kFastNp = 16;   // complex lines (row pairs) per CTA of a fast x pass

constexpr int fast_gcd(int a, int b) { return b == 0 ? a : fast_gcd(b, a % b); }
// threads of a fast pass CTA for `lines` lines: lines x the gcd of the stages'
// butterfly counts (so the trips divide evenly), brought into [64, 256] by
// powers of two
constexpr int fast_threads(int r1, int r2, int r3, int lines) {
    const int L = r1 * r2 * r3;
    int g = fast_gcd(L / r1, L / r2);
    if (r3 > 1) g = fast_gcd(g, L / r3);
    int nt = lines * g;
    while (nt < 64) nt *= 2;
    while (nt > 256 && nt % 2 == 0) nt /= 2;
    return nt;
}
// 1 when length L has a compile-time plan
inline bool fast_length(int L) {
#define APM_FAST_CASE(LL, A, B, C) if (L == LL) return true;
    APM_FAST_LENGTHS(APM_FAST_CASE)
#undef APM_FAST_CASE
    return false;
}
// dynamic shared memory of a fast column-pass CTA: the buffer and the twiddles
inline size_t fast_col_smem(int L) { return (size_t)(L * kFastTx + L) * sizeof(float2); }
// ... and of a fast x-pass CTA (rows padded to kFastNp + 1 lines)
// (the x-inverse pads its lines by one element every R_last positions: at
// most L / 2 more)
inline size_t fast_row_smem(int L) { return (size_t)(L * (kFastNp + 1) + L / 2 + L) * sizeof(float2); }

// Column-pass chunks carry (kx tile, line index of the other axis) as
// (kt << 20) | other: other < 2^20, kt < 2^11.
constexpr int kColOtherBits = 20;

// Everything a kernel needs to know about one grid.
struct GridDev {
    int kind;            // Green's table: 0 refined, 1 periodic root, 2 isolated root
    int mode;            // deposit edge rule: 0 drop, 1 fold, 2 wrap
    int N[3];            // interior cells
    int G[3];            // GMF box
    int M[3];            // FFT lengths
    int W[3];            // window N + 4 (cells [-2, N+2))
    int s0[3];           // M index of window cell -2, in [0, M)
    int Hx;              // M[0]/2 + 1 (half spectrum along x)
    int Hy2, Hz2;        // M[1]/2 + 1, M[2]/2 + 1 (octant table)
    long long lo[3];     // global level index of GMF cell 0
    long long start[3];  // global level index of interior cell 0
    int parent;          // index of the parent among the grids of level - 1, or -1
    int pN[3];
    long long pstart[3];
    double delta;
    FftPlan1D fx, fy, fz;
    FftPlan1D iy, iz;    // fy, fz with the radices reversed (inverse column transforms)
    long long tab_off;   // octant table offset (elements) in the table arenas
    long long wsA, wsB;  // workspace offsets (complex elements)
    long long cells_gmf; // G0 G1 G2
    int lines[kFftPasses];   // lines per CTA of each pass (row pairs for xf / xi)
    int rows_gas;        // GMF rows per CTA of the baryon initialisation
    int acc_sh[3];       // 1 when output cell 0 is the second cell of its block, else 0
    int acc_nb[3];       // output blocks per axis
    double inv2d;        // 1 / (2 delta)
    double inv_m3;       // 1 / (M0 M1 M2), the inverse transform's normalisation
    int grad;            // gradient operator (apm_gradient): 0 two-point, 1 four-point, 2 spectral
    int h;               // phi_short window half-width: cells [-h, N+h) (3 four-point, else 2)
    double dk[3];        // 2 pi / (M_j delta): the spectral gradient's k per mode index
    double inv12d;       // 1 / (12 delta)
};

// Threads of a CTA walking a batch of rows [r0, r1) of length n in row-major
// order: thread t starts at element t and strides by the block size, the
// (row, x) pair stepped incrementally (no division per element).
struct RowWalk {
    int r, x, dr, dx, n;
    __device__ RowWalk(int r0, int n_) : n(n_) {
        r = r0;
        x = threadIdx.x;
        while (x >= n) {
            x -= n;
            ++r;
        }
        dr = blockDim.x / n;
        dx = blockDim.x - dr * n;
    }
    __device__ void next() {
        x += dx;
        r += dr;
        if (x >= n) {
            x -= n;
            ++r;
        }
    }
};

// 2x2x2 output blocks per CTA of the acceleration kernel (flat ranges of the
// grid's blocks, x fastest, so every thread gets the same count)
constexpr int kAccBlocksPerCta = 512;

// Threads of a CTA walking the flat range [f0, f0 + count) of elements of rows
// of length n: thread t starts at f0 + t and strides by the block size, with
// (row, x) stepped incrementally (one division per thread).
struct FlatWalk {
    int r, x, dr, dx, n, left;
    __device__ FlatWalk(long long f0, int count, int n_) : n(n_) {
        const long long f = f0 + threadIdx.x;
        r = (int)(f / n);
        x = (int)(f - (long long)r * n);
        left = count - (int)threadIdx.x;
        dr = blockDim.x / n;
        dx = blockDim.x - dr * n;
    }
    __device__ bool ok() const { return left > 0; }
    __device__ void next() {
        left -= blockDim.x;
        x += dx;
        r += dr;
        if (x >= n) {
            x -= n;
            ++r;
        }
    }
};

// Tile lookup: level cell -> candidate grids (CSR per tile).
struct TileMap {
    long long lo[3];
    int shift;
    int nt[3];
    const int* dep_off;   // grids whose GMF box, grown by one cell, meets the tile
    const int* dep_list;
    const int* own_off;   // grids whose interior meets the tile
    const int* own_list;
    const unsigned char* occ;  // 1 if the tile or one of its 26 neighbours has a dep entry
};

struct Chunk { int grid; int tile; };   // one CTA of a batched pass

// Per-level device view (passed by value to kernels).
struct LevelDev {
    int level;
    int n;                 // grids on the level
    int is_root;
    int refine;
    const GridDev* g;      // n descriptors
    TileMap map;
    double delta;
    double inv_delta;      // 1/delta
    double delta0;         // root cell: fixed-point positions count 2^-31 root cells
    double inv_delta0;
    int delta0_pow2;       // delta0 is a power of two: x/delta0 == x*inv_delta0 exactly
    int frac_bits;         // 31 - level: fraction bits of a position on this level
    long long span;        // N0 2^31: the box in fixed-point units
    double box;
    int periodic;
    int pos_exp;           // delta0 = 2^(31 - pos_exp) when delta0_pow2: X = rint(x 2^pos_exp)
    unsigned* status;      // the context's device status word (bounds-checked builds)
};

// Fixed-point TSC (shared by the deposit and the interpolation).  A drifted
// coordinate x becomes X = rint(x/delta0 2^31) once; on a level with P fraction
// bits the cell is X >> P and t = (X mod 2^P)/2^P; the weights of cells i-1, i,
// i+1 are (1-t)^2/2, 3/4 - (t-1/2)^2, t^2/2 as exact integers on the scale 2^63.
constexpr int kPosBits = 31;
constexpr unsigned long long kOne63 = 1ULL << 63;

// rint(x 2^K), ties to even, of a finite double with |x 2^K| < 2^62, from its
// exponent and significand with integer operations (no FP64 pipe); ok is
// cleared for larger or non-finite values.
__device__ __forceinline__ long long scaled_rint(double x, int K, bool& ok) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    ok = true;
    if (e == 0x7FF) {
        ok = false;
        return 0;
    }
    if (e == 0) return 0;   // zero or subnormal: far below one unit here
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFULL) | 0x10000000000000ULL;
    const int sh = e - 1075 + K;   // |x 2^K| = m 2^sh
    unsigned long long r;
    if (sh >= 0) {
        if (sh >= 10) {            // m 2^sh >= 2^62
            ok = false;
            return 0;
        }
        r = m << sh;
    } else if (sh < -54) {
        r = 0;
    } else {
        const int t = -sh;
        r = m >> t;
        const unsigned long long rem = m & ((1ULL << t) - 1);
        const unsigned long long half = 1ULL << (t - 1);
        if (rem > half || (rem == half && (r & 1))) ++r;
    }
    return (b >> 63) ? -(long long)r : (long long)r;
}

// x' = x + v half_dt in FP64 (two rounded operations)
__device__ __forceinline__ double drift_raw(double x, double v, double half_dt) {
    return __dadd_rn(x, __dmul_rn(v, half_dt));
}

// X = rint(x'/delta0 2^31), canonical: modulo the box on a periodic domain; on
// an isolated domain a coordinate inside [0, box) that rounds onto the upper
// face stays in the last cell
__device__ __forceinline__ long long fixed_position(double xd, const LevelDev& L) {
    // a coordinate 2^31 root cells or more from the origin (or NaN) saturates at
    // -+2^62: far outside every box
    long long X;
    bool ok;
    if (L.delta0_pow2) {
        X = scaled_rint(xd, L.pos_exp, ok);
    } else {
        const double t = __dmul_rn(__ddiv_rn(xd, L.delta0), 2147483648.0);
        ok = fabs(t) < 4611686018427387904.0;   // 2^62
        X = ok ? __double2ll_rn(t) : 0;
    }
    if (!ok) X = xd > 0.0 ? (1LL << 62) : -(1LL << 62);
    if (L.periodic) {
        if (X < 0 || X >= L.span) {
            X %= L.span;
            if (X < 0) X += L.span;
        }
    } else if (X >= L.span && xd >= 0.0 && xd < L.box) {
        X = L.span - 1;
    }
    return X;
}

__device__ __forceinline__ long long tsc_fixed(long long X, int P, unsigned long long w[3]) {
    long long i = X >> P;
    unsigned f = (unsigned)(X - (i << P));
    unsigned S1 = (1u << P) - f;            // 2^P - f, at most 2^31
    const int up = 62 - 2 * P;
    w[2] = ((unsigned long long)f * f) << up;
    w[0] = ((unsigned long long)S1 * S1) << up;
    w[1] = kOne63 - w[0] - w[2];
    return i;
}

// (a b + 2^62) >> 63 for a, b < 2^63: product of two weights on the scale 2^63,
// rounded half up
__device__ __forceinline__ unsigned long long wmul63(unsigned long long a, unsigned long long b) {
    unsigned long long lo = a * b;
    unsigned long long hi = __umul64hi(a, b);
    unsigned long long lo2 = lo + (1ULL << 62);
    hi += (lo2 < lo) ? 1ULL : 0ULL;
    return (hi << 1) | (lo2 >> 63);
}

// ---- bulk asynchronous copies (TMA engine, no tensor map) and mbarriers ----
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barrier visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy of `bytes` (a multiple of 16; both addresses
// 16-byte aligned), completing on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// one poll of phase `parity`; a thread may be suspended up to kWaitHintNs
// nanoseconds inside it
constexpr unsigned kWaitHintNs = 1000;
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}
// waits for phase `parity` of `bar` at most `limit` polls (about a second in
// all); false when it ran out
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
constexpr unsigned kWaitPolls = 1u << 20;

// wmul63 for a < 2^32: with b = bh 2^32 + bl, (a b + 2^62) >> 63 equals
// (a bh + ((a bl) >> 32) + 2^30) >> 31 (the low 32 bits of a bl cannot carry
// into the result); two 32 x 32 -> 64 products
__device__ __forceinline__ unsigned long long wmul63_small(unsigned long long a, unsigned long long b) {
    const unsigned a32 = (unsigned)a;
    const unsigned long long hi = (unsigned long long)a32 * (unsigned)(b >> 32);
    const unsigned long long lo = (unsigned long long)a32 * (unsigned)b;
    return (hi + (lo >> 32) + (1ULL << 30)) >> 31;
}

struct Particles {
    long long n;
    const double *x, *y, *z, *vx, *vy, *vz, *m;
    const int* perm = nullptr;   // processing order (launch_order): slot i visits particle perm[i]
    int order_shift = 0;         // ... sorted by bins of 2^order_shift root cells (x fastest)
    __device__ __forceinline__ long long at(long long i) const { return perm ? (long long)perm[i] : i; }
};

// ---------------------------------------------------------------------------
// launchers (each returns the launch error)
// ---------------------------------------------------------------------------
// twiddles exp(-2 pi i t / L) for t < L, FP64 and FP32
cudaError_t launch_twiddles(double2* tw64, float2* tw32, int L, cudaStream_t s);

// Green's tables (FP64 octant), kind 0/1 directly, kind 2 from the real-space kernel
cudaError_t launch_green_table(int kind, const int M[3], double delta, double a_lev,
                               double a_par, int correction, int grad, double* out, double* scratch,
                               cudaStream_t s);
cudaError_t launch_to_f32(const double* in, float* out, long long n, cudaStream_t s);

// GMF: baryons (initialises every cell) then particles
cudaError_t launch_gas_init(const LevelDev& L, const GridDev* parent_grids,
                            const double* const* gas, const double* const* pgas,
                            int64_t* const* gmf, const Chunk* chunks, int n_chunks,
                            int F, cudaStream_t s);
cudaError_t launch_deposit(const LevelDev& L, const Particles& P, double half_dt, double box,
                           int F, int64_t* const* gmf, unsigned* status, cudaStream_t s);
// every level in one pass: levels[nl] and gmfs[nl] in device memory
cudaError_t launch_deposit_levels(const LevelDev* levels, int nl, const Particles& P, double half_dt,
                                  double box, int F, int64_t* const* const* gmfs, unsigned* status,
                                  cudaStream_t s);

// FFT passes of one level (T = float or double)
struct FftArgs {
    const GridDev* g;
    const Chunk* chunks;
    int n_chunks;
    const void* tw;        // complex twiddle arena of the precision
    const void* tab;       // table arena of the precision
    void* wsA;
    void* wsB;
    int F;
    size_t smem;
    int threads;           // threads per CTA: 128 or 256
    unsigned* status;      // device status word (bounded waits that ran out), or null
    int inject_wait = 0;   // fault injection: the x-forward bulk copy's wait runs out
    int comp = 0;          // spectral gradient: component of the z / xi passes (0 phi, 1-3 A_x..A_z)
};
cudaError_t fft_configure();

// Particle processing order (k_order.cu): a counting sort of the particle
// indices by root-level bin (cubes of 2^shift root cells, nb bins per axis) of
// their drifted positions into perm; count holds nb^3 bins, sums
// order_scan_chunks(nb^3) <= 1024 entries, key and rank n entries each.
int order_scan_chunks(int nbins);
cudaError_t launch_order(const LevelDev& root, const Particles& P, double half_dt, int shift, int nb,
                         unsigned* count, unsigned* sums, unsigned* key, unsigned* rank, int* perm, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_xf(const FftArgs& a, const int64_t* const* gmf, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_yf(const FftArgs& a, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_z(const FftArgs& a, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_yi(const FftArgs& a, cudaStream_t s);
// the z pass of a spectral-gradient component (a.comp in 1..3): the table
// times -i D_comp between the forward and the inverse transform
template <typename T>
cudaError_t launch_fft_zgrad(const FftArgs& a, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_xi(const FftArgs& a, void* const* phis, cudaStream_t s);
// FP32 column passes of length L with a compile-time plan (fast_length(L)):
// yf, z (with the table) and yi; a.chunks hold kFastTx columns per CTA
cudaError_t launch_fft_yf_fast(int L, const FftArgs& a, cudaStream_t s);
cudaError_t launch_fft_z_fast(int L, const FftArgs& a, cudaStream_t s);
cudaError_t launch_fft_zgrad_fast(int L, const FftArgs& a, cudaStream_t s);   // spectral component a.comp
cudaError_t launch_fft_yi_fast(int L, const FftArgs& a, cudaStream_t s);
// the fused x + y forward over one z plane (k_xy_fast) of a grid with
// M0 = M1 = L: the plane (L rows x L/2 + 1 columns) and the twiddles
constexpr int kFastXyThreads = 384;
inline size_t fast_xy_smem(int L) { return (size_t)(L * (L / 2 + 1) + L) * sizeof(float2); }
inline bool fast_xy_length(int L) { return fast_length(L) && fast_xy_smem(L) <= (size_t)kFftSmemLimit; }
cudaError_t launch_fft_xy_fast(int L, const FftArgs& a, const int64_t* const* gmf, cudaStream_t s);
// ... and its inverse, the fused y + x inverse over one window plane
// (k_yx_fast), for grids whose window fits the transform (W1 <= M1)
cudaError_t launch_fft_yx_fast(int L, const FftArgs& a, void* const* phis, cudaStream_t s);

// FP32 x passes of length M0 = L with a compile-time plan: kFastNp row pairs
// per CTA (both use fast_row_smem)
cudaError_t launch_fft_xf_fast(int L, const FftArgs& a, const int64_t* const* gmf, cudaStream_t s);
cudaError_t launch_fft_xi_fast(int L, const FftArgs& a, void* const* phis, cudaStream_t s);

// accelerations + parent carry for the four-point and spectral gradients (the
// two-point one runs launch_accel), on launch_accel's block work list
template <typename T>
cudaError_t launch_accel_var(const LevelDev& L, const GridDev* parent_grids, const void* const* phis,
                               const void* const* pphi, const void* const* pacc, void* const* phi,
                               void* const* acc, const Chunk* chunks, int n_chunks, int grad,
                               cudaStream_t s);

// FD accelerations + parent carry; TSC interpolation
template <typename T>
cudaError_t launch_accel(const LevelDev& L, const GridDev* parent_grids, const void* const* phis,
                         const void* const* pphi, const void* const* pacc, void* const* phi,
                         void* const* acc, const Chunk* chunks, int n_chunks,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_interp(const LevelDev& L, const LevelDev* finer, const Particles& P,
                          double half_dt, const void* const* acc, void* out, cudaStream_t s);
// every level in one pass: levels[nl] and accs[nl] in device memory
template <typename T>
cudaError_t launch_interp_levels(const LevelDev* levels, int nl, const Particles& P, double half_dt,
                                 const void* const* const* accs, void* out, cudaStream_t s);

// one leapfrog step of the particles (k_evolve.cu); acc: 3n values of T
template <typename T>
cudaError_t launch_kick_drift(long long n, double* x, double* y, double* z, double* vx, double* vy, double* vz,
                              const void* acc, double dt, cudaStream_t s);

}  // namespace apm

// apm_noalloc.cu -- apm_solve_periodic_noalloc: the potential solve of one
// periodic root grid that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: applications that give the whole device
// to their own memory pool at start-up, so that a library allocating behind
// their back would fail or break the pool's accounting, and loops that must
// not stall on the device-wide synchronisation cudaFree implies.  This entry
// point needs no context and no allocation: every intermediate it uses
// (twiddles, the Green's table, grid descriptors, a status word and the two
// spectrum buffers of the FFT passes) lives in one fixed, file-scope device
// array, kScratchBytes large, that every GPU which loads the library holds
// until the process exits.
#include <algorithm>
#include <cstring>

#include "apm_internal.cuh"

namespace apm {
namespace {

constexpr int kNoallocMaxN = 128;                        // largest grid: 128^3
constexpr size_t kScratchBytes = 24u << 20;              // 24 MiB
constexpr int kMaxChunks = 8192;
constexpr int kMaxDevices = 64;

// The scratch.  In host code this name is only a host-side stand-in for the
// device array; host code must use the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

void* g_scratch_addr[kMaxDevices] = {};

// writes the descriptor, the pointer tables of the passes and a chunk list
// {grid 0, tile i} into the scratch
// row chunks {0, i}; column chunks {0, (kt << kColOtherBits) | other} for
// i = other * nkt + kt
// (and clears the status word the x-forward pass's bounded wait reports to)
__global__ void k_noalloc_setup(GridDev g, GridDev* dst, Chunk* chunks, Chunk* cchunks, int n, int nkt,
                                const int64_t** in_tab, const int64_t* in, void** out_tab, void* out,
                                unsigned* status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *dst = g;
        *in_tab = in;
        *out_tab = out;
        *status = 0u;
    }
    if (i < n) {
        chunks[i] = Chunk{0, i};
        const int other = i / nkt, kt = i - other * nkt;
        cchunks[i] = Chunk{0, (kt << kColOtherBits) | other};
    }
}

// There is no status reader for this entry point, so a wait that ran out must
// show in the output itself: if the status word is set, the whole window is
// overwritten with NaN.  One CTA; it reads one word and returns when it is 0.
__global__ void k_noalloc_finish(const unsigned* status, float* out, long long count) {
    if (*status == 0u) return;
    const float nan = __int_as_float(0x7fc00000);
    for (long long i = threadIdx.x; i < count; i += blockDim.x) out[i] = nan;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace apm

using namespace apm;

extern "C" apm_status apm_solve_periodic_noalloc(int32_t n, double box, double a_over_dx,
                                                 int32_t mass_frac_bits, const int64_t* gmf,
                                                 float* phi_short, void* stream) {
    if (n < 4 || n > kNoallocMaxN || !(box > 0) || !(a_over_dx > 0) || mass_frac_bits < 1 ||
        mass_frac_bits > 62 || !gmf || !phi_short)
        return APM_E_INVALID;
    GridDev g;
    std::memset(&g, 0, sizeof(g));
    if (!fft_plan(n, 16, &g.fx)) return APM_E_INVALID;   // n must be {2,3,5,7}-smooth
    g.fy = g.fx;
    g.fz = g.fx;
    fft_plan_reversed(g.fx, &g.iy);
    g.iz = g.iy;
    cudaStream_t s = (cudaStream_t)stream;

    // set-up, once per device, with that device current: the scratch address
    // and the shared-memory limit of the FFT kernels
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return APM_E_CUDA;
    }
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return APM_E_CUDA;
        }
        if (fft_configure() != cudaSuccess) return APM_E_CUDA;
        g_scratch_addr[dev] = p;
    }
    unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);

    // the grid: periodic root, M = N = n, window [-2, n+2)
    const double delta = box / n;
    g.kind = 1;
    g.mode = 2;
    for (int j = 0; j < 3; ++j) {
        g.N[j] = g.G[j] = g.M[j] = n;
        g.W[j] = n + 4;
        g.s0[j] = n - 2;
    }
    g.Hx = g.Hy2 = g.Hz2 = n / 2 + 1;
    g.delta = delta;
    g.parent = -1;
    g.cells_gmf = (long long)n * n * n;
    g.inv_m3 = 1.0 / ((double)n * (double)n * (double)n);
    for (int q = 0; q < kFftPasses; ++q) g.lines[q] = fft_pass_lines(q, n, kFftBudgetF32, false);
    const long long Hx = g.Hx;
    const long long szA = (long long)(n + 4) * n * Hx;         // max(G1 G2, W2 M1) Hx
    const long long szB = (long long)(n + 4) * (n + 4) * Hx;   // max(G2 M1, W2 W1) Hx
    const long long tab = Hx * Hx * Hx;

    // scratch layout
    size_t off = 0;
    GridDev* d_g = reinterpret_cast<GridDev*>(base + off);
    off = align256(off + sizeof(GridDev));
    unsigned* d_status = reinterpret_cast<unsigned*>(base + off);
    off = align256(off + sizeof(unsigned));
    Chunk* d_chunks = reinterpret_cast<Chunk*>(base + off);
    off = align256(off + kMaxChunks * sizeof(Chunk));
    Chunk* d_cchunks = reinterpret_cast<Chunk*>(base + off);
    off = align256(off + kMaxChunks * sizeof(Chunk));
    double2* tw64 = reinterpret_cast<double2*>(base + off);
    off = align256(off + n * sizeof(double2));
    float2* tw32 = reinterpret_cast<float2*>(base + off);
    off = align256(off + n * sizeof(float2));
    double* tab64 = reinterpret_cast<double*>(base + off);
    off = align256(off + tab * sizeof(double));
    float* tab32 = reinterpret_cast<float*>(base + off);
    off = align256(off + tab * sizeof(float));
    float2* wsA = reinterpret_cast<float2*>(base + off);
    off = align256(off + szA * sizeof(float2));
    float2* wsB = reinterpret_cast<float2*>(base + off);
    off = align256(off + szB * sizeof(float2));
    if (off > kScratchBytes) return APM_E_INVALID;
    g.fx.tw_off = g.fy.tw_off = g.fz.tw_off = 0;
    g.tab_off = 0;
    g.wsA = 0;
    g.wsB = 0;

    // CTAs of each pass (one grid)
    const int nky = (int)((Hx + g.lines[kPassYf] - 1) / g.lines[kPassYf]);   // the same for yi and z
    const long long pairs_in = ((long long)n * n + 1) / 2;
    const long long pairs_out = ((long long)(n + 4) * (n + 4) + 1) / 2;
    const int n_xf = (int)((pairs_in + g.lines[kPassXf] - 1) / g.lines[kPassXf]);
    const int n_yf = nky * n;
    const int n_z = nky * n;
    const int n_yi = nky * (n + 4);
    const int n_xi = (int)((pairs_out + g.lines[kPassXi] - 1) / g.lines[kPassXi]);
    const int n_max = std::max(std::max(n_xf, n_yf), std::max(std::max(n_z, n_yi), n_xi));
    if (n_max > kMaxChunks - 2) return APM_E_INVALID;
    // the per-grid pointer tables of the passes sit in the last two chunk slots
    const int64_t** d_in = reinterpret_cast<const int64_t**>(d_chunks + (kMaxChunks - 2));
    void** d_out = reinterpret_cast<void**>(d_chunks + (kMaxChunks - 1));

    // every call rebuilds what it reads (and clears the status word): nothing
    // depends on the previous call
    k_noalloc_setup<<<(n_max + 255) / 256, 256, 0, s>>>(g, d_g, d_chunks, d_cchunks, n_max, nky, d_in, gmf,
                                                        d_out, phi_short, d_status);
    if (cudaGetLastError() != cudaSuccess) return APM_E_CUDA;
    if (launch_twiddles(tw64, tw32, n, s) != cudaSuccess) return APM_E_CUDA;
    const int M[3] = {n, n, n};
    if (launch_green_table(1, M, delta, a_over_dx * delta, 0.0, 0, APM_GRAD_FD2, tab64, nullptr, s) != cudaSuccess)
        return APM_E_CUDA;
    if (launch_to_f32(tab64, tab32, tab, s) != cudaSuccess) return APM_E_CUDA;

    FftArgs a;
    a.g = d_g;
    a.chunks = d_chunks;
    a.tw = tw32;
    a.tab = tab32;
    a.wsA = wsA;
    a.wsB = wsB;
    a.F = mass_frac_bits;
    a.threads = kFftThreads;
    a.status = d_status;  // read by k_noalloc_finish after the last pass
    const size_t smem_rows = fft_pass_smem(kPassXf, n, g.lines[kPassXf], sizeof(float2), n);
    const size_t smem_cols = fft_pass_smem(kPassYf, n, g.lines[kPassYf], sizeof(float2));
    a.n_chunks = n_xf;
    a.smem = smem_rows;
    if (launch_fft_xf<float>(a, d_in, s) != cudaSuccess) return APM_E_CUDA;
    a.chunks = d_cchunks;
    a.n_chunks = n_yf;
    a.smem = smem_cols;
    if (launch_fft_yf<float>(a, s) != cudaSuccess) return APM_E_CUDA;
    a.n_chunks = n_z;
    if (launch_fft_z<float>(a, s) != cudaSuccess) return APM_E_CUDA;
    a.n_chunks = n_yi;
    if (launch_fft_yi<float>(a, s) != cudaSuccess) return APM_E_CUDA;
    a.chunks = d_chunks;
    a.n_chunks = n_xi;
    a.smem = smem_rows;
    if (launch_fft_xi<float>(a, d_out, s) != cudaSuccess) return APM_E_CUDA;
    k_noalloc_finish<<<1, 256, 0, s>>>(d_status, phi_short, (long long)(n + 4) * (n + 4) * (n + 4));
    if (cudaGetLastError() != cudaSuccess) return APM_E_CUDA;
    return APM_OK;
}

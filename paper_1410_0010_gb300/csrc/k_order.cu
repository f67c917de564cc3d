// k_order.cu -- a spatially coherent processing order of the particles: a
// counting sort of the particle indices by the root-level bin (cubes of 2^shift
// root cells) of their drifted positions.  The interpolation kernels then visit
// the particles bin by bin, so a warp's clouds overlap and its gathers touch
// the same cache lines.  The order changes no result: each particle is
// interpolated on its own.
#include "apm_internal.cuh"

namespace apm {
namespace {

constexpr int kScanChunk = 2048;   // bins per CTA of the local scan (1024 threads x 2)

// bin of each particle and its rank inside the bin (the count before it)
__global__ void __launch_bounds__(256) k_order_bins(LevelDev L, Particles P, double half_dt, int shift, int nb,
                                                    unsigned* __restrict__ count, unsigned* __restrict__ key,
                                                    unsigned* __restrict__ rank) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P.n) return;
    const double xd[3] = {drift_raw(P.x[p], P.vx[p], half_dt), drift_raw(P.y[p], P.vy[p], half_dt),
                          drift_raw(P.z[p], P.vz[p], half_dt)};
    long long b[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const long long ic = fixed_position(xd[j], L) >> L.frac_bits;   // root cell (may be outside)
        const long long v = ic >> shift;
        b[j] = v < 0 ? 0 : (v >= nb ? nb - 1 : v);
    }
    const unsigned k = (unsigned)(b[0] + (long long)nb * (b[1] + (long long)nb * b[2]));
    key[p] = k;
    rank[p] = atomicAdd(count + k, 1u);
}

// exclusive scan of each chunk of kScanChunk counts in place; the chunk's total
// to sums[chunk]
__global__ void __launch_bounds__(1024) k_order_scan_local(unsigned* __restrict__ count, int nbins,
                                                           unsigned* __restrict__ sums) {
    __shared__ unsigned warp_tot[32];
    const int base = blockIdx.x * kScanChunk + 2 * threadIdx.x;
    const unsigned a = base < nbins ? count[base] : 0u;
    const unsigned b = base + 1 < nbins ? count[base + 1] : 0u;
    const unsigned t = a + b;
    // inclusive scan of t over the CTA: warp shuffles, then the warp totals
    unsigned v = t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned w = warp_tot[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += u;
        }
        warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const unsigned before = v - t + (warp > 0 ? warp_tot[warp - 1] : 0u);   // exclusive prefix of a
    if (base < nbins) count[base] = before;
    if (base + 1 < nbins) count[base + 1] = before + a;
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = before + t;
}

// exclusive scan of the chunk totals (at most 1024 chunks) in place, one CTA
__global__ void __launch_bounds__(1024) k_order_scan_sums(unsigned* __restrict__ sums, int n) {
    __shared__ unsigned warp_tot[32];
    const unsigned t = threadIdx.x < (unsigned)n ? sums[threadIdx.x] : 0u;
    unsigned v = t;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned w = warp_tot[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += u;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)n) sums[threadIdx.x] = v - t + (warp > 0 ? warp_tot[warp - 1] : 0u);
}

// perm[slot] = p with slot = (chunk offset + bin offset + rank)
__global__ void __launch_bounds__(256) k_order_scatter(long long n, const unsigned* __restrict__ key,
                                                       const unsigned* __restrict__ rank,
                                                       const unsigned* __restrict__ count,
                                                       const unsigned* __restrict__ sums, int* __restrict__ perm) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const unsigned k = key[p];
    const unsigned slot = sums[k / kScanChunk] + count[k] + rank[p];
    perm[slot] = (int)p;
}

}  // namespace

int order_scan_chunks(int nbins) { return (nbins + kScanChunk - 1) / kScanChunk; }

cudaError_t launch_order(const LevelDev& root, const Particles& P, double half_dt, int shift, int nb,
                         unsigned* count, unsigned* sums, unsigned* key, unsigned* rank, int* perm, cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    const int nbins = nb * nb * nb;
    const int nchunks = order_scan_chunks(nbins);
    if (nchunks > 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(count, 0, (size_t)nbins * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((P.n + 255) / 256);
    k_order_bins<<<blocks, 256, 0, s>>>(root, P, half_dt, shift, nb, count, key, rank);
    k_order_scan_local<<<nchunks, 1024, 0, s>>>(count, nbins, sums);
    k_order_scan_sums<<<1, 1024, 0, s>>>(sums, nchunks);
    k_order_scatter<<<blocks, 256, 0, s>>>(P.n, key, rank, count, sums, perm);
    return cudaGetLastError();
}

}  // namespace apm

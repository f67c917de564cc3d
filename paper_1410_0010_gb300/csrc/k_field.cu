// k_field.cu -- cell accelerations with the parent carry, and TSC interpolation
// of the accelerations back to the particles (Sec. 2.2, Sec. 2).
#include "apm_internal.cuh"

namespace apm {
namespace {

// Trilinear weights of child cell ic from the parent cell centres, R = 2: in
// parent units the child centre is at (ic + 1/2)/2, i.e. 3/4 (even ic) or 1/4
// (odd ic) of a cell above the centre of parent cell i0 = floor((ic - 1) / 2),
// so i0 weighs 1/4 for even ic and 3/4 for odd ic (i0 + 1 the rest).
__device__ __forceinline__ void carry_axis(long long ic, long long pstart, int& i0, float& w_lo) {
    long long a = (ic - 1) >> 1;          // floor((ic - 1) / 2)
    i0 = (int)(a - pstart) + 1;           // +1: parent ghost offset
    w_lo = (ic & 1) ? 0.75f : 0.25f;
}

// trilinear interpolation of one parent field, separably (x, then y, then z);
// the weights 1/4, 3/4 are exact in either precision
template <typename T>
__device__ __forceinline__ T trilinear(const T* __restrict__ f, unsigned base, int P0, unsigned P01,
                                       T wx, T wy, T wz) {
    T c[2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const T* r = f + base + dy * P0 + dz * P01;
            c[dz][dy] = wx * r[0] + ((T)1 - wx) * r[1];
        }
    T e0 = wy * c[0][0] + ((T)1 - wy) * c[0][1];
    T e1 = wy * c[1][0] + ((T)1 - wy) * c[1][1];
    return wz * e0 + ((T)1 - wz) * e1;
}

// acc_j(c) = -(phis(c+e_j) - phis(c-e_j)) / (2 delta) + I(parent acc_j)(c)
// phi(c)   = phis(c) + I(parent phi)(c),    c in [-1, N]^3
// I is the trilinear interpolation from the parent cell centres.  Everything is
// evaluated in T: the FP64 path in FP64, the FP32 path in FP32 (the weights are
// exact; the interpolated FP32 fields carry no more digits than FP32 anyway).
// One CTA per batch of `rows_per_cta` output rows (x fastest over threads).
template <typename T>
__global__ void __launch_bounds__(256) k_accel(LevelDev L, const GridDev* __restrict__ pgrids,
                                               const void* const* __restrict__ phis_p,
                                               const void* const* __restrict__ pphi_p,
                                               const void* const* __restrict__ pacc_p,
                                               void* const* __restrict__ phi_p,
                                               void* const* __restrict__ acc_p,
                                               const Chunk* __restrict__ chunks, int rows_per_cta) {
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = L.g[ch.grid];
    const int E0 = g.N[0] + 2, E1 = g.N[1] + 2, E2 = g.N[2] + 2;
    const unsigned ncell = (unsigned)E0 * E1 * E2;
    const int nrows = E1 * E2;
    const int W0 = g.W[0], W1 = g.W[1];
    const T* __restrict__ phis = reinterpret_cast<const T*>(phis_p[ch.grid]);
    T* __restrict__ phi = reinterpret_cast<T*>(phi_p[ch.grid]);
    T* __restrict__ acc = reinterpret_cast<T*>(acc_p[ch.grid]);
    const bool carry = pphi_p != nullptr && g.parent >= 0;
    const T* __restrict__ pphi = carry ? reinterpret_cast<const T*>(pphi_p[g.parent]) : nullptr;
    const T* __restrict__ pacc = carry ? reinterpret_cast<const T*>(pacc_p[g.parent]) : nullptr;
    int P0 = 0;
    unsigned P01 = 0, pn = 0;
    long long ps0 = 0, ps1 = 0, ps2 = 0;
    if (carry) {
        const GridDev& p = pgrids[g.parent];
        P0 = p.N[0] + 2;
        P01 = (unsigned)P0 * (p.N[1] + 2);
        pn = P01 * (p.N[2] + 2);
        ps0 = p.start[0]; ps1 = p.start[1]; ps2 = p.start[2];
    }
    const T inv2d = (T)g.inv2d;
    const unsigned sy = W0, sz = (unsigned)W0 * W1;
    const int r0 = ch.tile * g.rows_acc;
    const int r1 = min(nrows, r0 + g.rows_acc);
    int last = -1, iy = 0, iz = 0;
    float wyf = 0.f, wzf = 0.f;
    unsigned prow = 0, orow = 0;
    for (RowWalk it(r0, E0); it.r < r1; it.next()) {
        const int r = it.r, ex = it.x;
        if (r != last) {
            last = r;
            const int ey = r % E1, ez = r / E1;
            if (carry) {
                carry_axis(g.start[1] + (long long)ey - 1, ps1, iy, wyf);
                carry_axis(g.start[2] + (long long)ez - 1, ps2, iz, wzf);
            }
            prow = 1 + sy * (ey + 1) + sz * (ez + 1);   // phis index of x = -1
            orow = (unsigned)r * E0;
        }
        const unsigned ps = prow + ex;
        T p0 = phis[ps];
        T a0 = -(phis[ps + 1] - phis[ps - 1]) * inv2d;
        T a1 = -(phis[ps + sy] - phis[ps - sy]) * inv2d;
        T a2 = -(phis[ps + sz] - phis[ps - sz]) * inv2d;
        if (carry) {
            int ix;
            float wxf;
            carry_axis(g.start[0] + (long long)ex - 1, ps0, ix, wxf);
            const unsigned base = ix + P0 * iy + P01 * iz;
            const T wx = (T)wxf, wy = (T)wyf, wz = (T)wzf;
            p0 += trilinear<T>(pphi, base, P0, P01, wx, wy, wz);
            a0 += trilinear<T>(pacc, base, P0, P01, wx, wy, wz);
            a1 += trilinear<T>(pacc + pn, base, P0, P01, wx, wy, wz);
            a2 += trilinear<T>(pacc + 2 * pn, base, P0, P01, wx, wy, wz);
        }
        const unsigned o = orow + ex;
        phi[o] = p0;
        acc[o] = a0;
        acc[ncell + o] = a1;
        acc[2 * ncell + o] = a2;
    }
}


// index of the grid of level L whose interior holds level cell ic, or -1
__device__ int find_owner(const LevelDev& L, const long long ic[3]) {
    if (L.is_root) {
        const GridDev& g = L.g[0];
        for (int j = 0; j < 3; ++j)
            if (ic[j] < 0 || ic[j] >= g.N[j]) return -1;
        return 0;
    }
    const TileMap& m = L.map;
    long long t[3];
    for (int j = 0; j < 3; ++j) {
        long long rel = ic[j] - m.lo[j];
        if (rel < 0) return -1;
        t[j] = rel >> m.shift;
        if (t[j] >= m.nt[j]) return -1;
    }
    long long tile = t[0] + (long long)m.nt[0] * (t[1] + (long long)m.nt[1] * t[2]);
    for (int e = m.own_off[tile]; e < m.own_off[tile + 1]; ++e) {
        int gi = m.own_list[e];
        const GridDev& g = L.g[gi];
        bool in = true;
        for (int j = 0; j < 3; ++j)
            if (ic[j] < g.start[j] || ic[j] >= g.start[j] + g.N[j]) in = false;
        if (in) return gi;
    }
    return -1;
}

template <typename T> __device__ __forceinline__ T weight63(unsigned long long W);
template <> __device__ __forceinline__ double weight63<double>(unsigned long long W) {
    return __ull2double_rn(W) * 1.0842021724855044e-19;    // 2^-63
}
template <> __device__ __forceinline__ float weight63<float>(unsigned long long W) {
    return __uint2float_rn((unsigned)(W >> 39)) * 5.9604644775390625e-08f;   // 2^-24
}

// TSC interpolation with the deposit's fixed-point weights: the 26 outer
// weights are the rounded products ((wx wy) wz), the centre weight is one minus
// their sum, exactly as the deposit distributes a particle's mass.
template <typename T>
__global__ void __launch_bounds__(256) k_interp(LevelDev L, LevelDev F, int has_finer, Particles P,
                                                double half_dt, double box, int periodic,
                                                const void* const* __restrict__ acc_p,
                                                T* __restrict__ out) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P.n) return;
    long long X[3];
    X[0] = fixed_position(drift_raw(P.x[p], P.vx[p], half_dt), L);
    X[1] = fixed_position(drift_raw(P.y[p], P.vy[p], half_dt), L);
    X[2] = fixed_position(drift_raw(P.z[p], P.vz[p], half_dt), L);
    long long ic[3];
    for (int j = 0; j < 3; ++j) ic[j] = X[j] >> L.frac_bits;
    int gi = find_owner(L, ic);
    if (gi < 0) return;
    if (has_finer) {
        long long fc[3];
        for (int j = 0; j < 3; ++j) fc[j] = X[j] >> F.frac_bits;
        if (find_owner(F, fc) >= 0) return;
    }
    unsigned long long w[3][3];
    for (int j = 0; j < 3; ++j) tsc_fixed(X[j], L.frac_bits, w[j]);
    unsigned long long wq[3][3][3];
    unsigned long long wsum = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == 1 && b == 1 && c == 1) {
                    wq[c][b][a] = 0;
                    continue;
                }
                wq[c][b][a] = wmul63(wmul63(w[0][a], w[1][b]), w[2][c]);
                wsum += wq[c][b][a];
            }
        }
    wq[1][1][1] = kOne63 - wsum;
    const GridDev& g = L.g[gi];
    const T* __restrict__ A = reinterpret_cast<const T*>(acc_p[gi]);
    const int E0 = g.N[0] + 2, E1 = g.N[1] + 2;
    const unsigned ncell = (unsigned)E0 * E1 * (g.N[2] + 2);
    const bool fold = g.mode == 1;
    int lc[3];
    for (int j = 0; j < 3; ++j) lc[j] = (int)(ic[j] - g.start[j]);
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int z = lc[2] + c - 1;
        if (fold) z = z < 0 ? 0 : (z >= g.N[2] ? g.N[2] - 1 : z);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            int y = lc[1] + b - 1;
            if (fold) y = y < 0 ? 0 : (y >= g.N[1] ? g.N[1] - 1 : y);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int x = lc[0] + a - 1;
                if (fold) x = x < 0 ? 0 : (x >= g.N[0] ? g.N[0] - 1 : x);
                const T wt = weight63<T>(wq[c][b][a]);
                unsigned idx = (unsigned)(x + 1) + (unsigned)E0 * ((unsigned)(y + 1) + (unsigned)E1 * (unsigned)(z + 1));
                a0 += wt * A[idx];
                a1 += wt * A[ncell + idx];
                a2 += wt * A[2 * ncell + idx];
            }
        }
    }
    out[p] = a0;
    out[P.n + p] = a1;
    out[2 * P.n + p] = a2;
}

}  // namespace

template <typename T>
cudaError_t launch_accel(const LevelDev& L, const GridDev* parent_grids, const void* const* phis,
                         const void* const* pphi, const void* const* pacc, void* const* phi,
                         void* const* acc, const Chunk* chunks, int n_chunks, int rows_per_cta,
                         cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    k_accel<T><<<n_chunks, 256, 0, s>>>(L, parent_grids, phis, pphi, pacc, phi, acc, chunks,
                                        rows_per_cta);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interp(const LevelDev& L, const LevelDev* finer, const Particles& P,
                          double half_dt, double box, int periodic, const void* const* acc,
                          void* out, cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((P.n + 255) / 256);
    LevelDev F = finer ? *finer : L;
    k_interp<T><<<blocks, 256, 0, s>>>(L, F, finer ? 1 : 0, P, half_dt, box, periodic, acc,
                                       reinterpret_cast<T*>(out));
    return cudaGetLastError();
}

template cudaError_t launch_accel<float>(const LevelDev&, const GridDev*, const void* const*,
                                         const void* const*, const void* const*, void* const*,
                                         void* const*, const Chunk*, int, int, cudaStream_t);
template cudaError_t launch_accel<double>(const LevelDev&, const GridDev*, const void* const*,
                                          const void* const*, const void* const*, void* const*,
                                          void* const*, const Chunk*, int, int, cudaStream_t);
template cudaError_t launch_interp<float>(const LevelDev&, const LevelDev*, const Particles&, double,
                                          double, int, const void* const*, void*, cudaStream_t);
template cudaError_t launch_interp<double>(const LevelDev&, const LevelDev*, const Particles&, double,
                                           double, int, const void* const*, void*, cudaStream_t);

}  // namespace apm

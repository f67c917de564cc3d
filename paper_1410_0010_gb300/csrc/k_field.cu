// k_field.cu -- cell accelerations with the parent carry, and TSC interpolation
// of the accelerations back to the particles (Sec. 2.2, Sec. 2).
#include "apm_internal.cuh"

namespace apm {
namespace {

// acc_j(c) = -(phis(c+e_j) - phis(c-e_j)) / (2 delta) + I(parent acc_j)(c)
// phi(c)   = phis(c) + I(parent phi)(c),    c in [-1, N]^3
// I is the trilinear interpolation from the parent cell centres (Sec. 2.2), for
// R = 2: level cells 2k+1 and 2k+2 lie 1/4 and 3/4 of a parent cell above the
// centre of parent cell k, so they weigh parent cells (k, k+1) with (3/4, 1/4)
// and (1/4, 3/4).  Each thread computes one 2x2x2 block of such cells: the 8
// parent values of a field serve all 8 cells, interpolated separably (x, then
// y, then z), and the 32 values of phis around the block serve the 8 centred
// differences.  Everything is evaluated in T; the weights are exact.
// A block may straddle the edge of [-1, N]: its outside cells are not written
// and the loads they would need are clamped into the window.
template <typename T>
__device__ __forceinline__ void lerp_block(const T q[2][2][2], T out[2][2][2]) {
    const T a = (T)0.75, b = (T)0.25;
    T x[2][2][2], y[2][2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            x[dz][dy][0] = a * q[dz][dy][0] + b * q[dz][dy][1];
            x[dz][dy][1] = b * q[dz][dy][0] + a * q[dz][dy][1];
        }
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
            y[dz][0][cx] = a * x[dz][0][cx] + b * x[dz][1][cx];
            y[dz][1][cx] = b * x[dz][0][cx] + a * x[dz][1][cx];
        }
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
            out[0][cy][cx] = a * y[0][cy][cx] + b * y[1][cy][cx];
            out[1][cy][cx] = b * y[0][cy][cx] + a * y[1][cy][cx];
        }
}

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }

template <typename T>
__device__ __forceinline__ void load_parent(const T* __restrict__ f, unsigned base, int P0, unsigned P01,
                                            T q[2][2][2]) {
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) q[dz][dy][dx] = f[base + dx + dy * P0 + dz * P01];
}

// CTA size and minimum resident CTAs per SM of the FP32 acceleration kernel
#ifndef APM_ACC_THREADS
#define APM_ACC_THREADS 128
#endif
#ifndef APM_ACC_MIN_CTAS
#define APM_ACC_MIN_CTAS 6
#endif
constexpr int kAccThreads = APM_ACC_THREADS;
template <typename T> struct AccMinCtas { static constexpr int value = APM_ACC_MIN_CTAS; };
template <> struct AccMinCtas<double> { static constexpr int value = 1; };

template <typename T>
__global__ void __launch_bounds__(kAccThreads, AccMinCtas<T>::value) k_accel(LevelDev L, const GridDev* __restrict__ pgrids,
                                               const void* const* __restrict__ phis_p,
                                               const void* const* __restrict__ pphi_p,
                                               const void* const* __restrict__ pacc_p,
                                               void* const* __restrict__ phi_p,
                                               void* const* __restrict__ acc_p,
                                               const Chunk* __restrict__ chunks) {
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = L.g[ch.grid];
    const int E0 = g.N[0] + 2, E1 = g.N[1] + 2, E2 = g.N[2] + 2;
    const unsigned ncell = (unsigned)E0 * E1 * E2;
    const int W0 = g.W[0], W1 = g.W[1], W2 = g.W[2];
    const int nbx = g.acc_nb[0], nby = g.acc_nb[1];
    const int nbrows = nby * g.acc_nb[2];
    const T* __restrict__ phis = reinterpret_cast<const T*>(phis_p[ch.grid]);
    T* __restrict__ phi = reinterpret_cast<T*>(phi_p[ch.grid]);
    T* __restrict__ acc = reinterpret_cast<T*>(acc_p[ch.grid]);
    const bool carry = pphi_p != nullptr && g.parent >= 0;
    const T* __restrict__ pphi = carry ? reinterpret_cast<const T*>(pphi_p[g.parent]) : nullptr;
    const T* __restrict__ pacc = carry ? reinterpret_cast<const T*>(pacc_p[g.parent]) : nullptr;
    int P0 = 0;
    unsigned P01 = 0, pn = 0;
    long long ps[3] = {0, 0, 0};
    if (carry) {
        const GridDev& p = pgrids[g.parent];
        P0 = p.N[0] + 2;
        P01 = (unsigned)P0 * (p.N[1] + 2);
        pn = P01 * (p.N[2] + 2);
        ps[0] = p.start[0]; ps[1] = p.start[1]; ps[2] = p.start[2];
    }
    const T inv2d = (T)g.inv2d;
    const unsigned sy = W0, sz = (unsigned)W0 * W1;
    const long long nblocks = (long long)nbx * nbrows;
    const long long f0 = (long long)ch.tile * kAccBlocksPerCta;
    const int count = (int)min((long long)kAccBlocksPerCta, nblocks - f0);
    // pair loads and stores need even row lengths and pointers aligned to two elements
    using V2 = typename Cplx<T>::type;
    const size_t amask = 2 * sizeof(T) - 1;
    const bool valign = !(W0 & 1) && !(E0 & 1) && !(reinterpret_cast<size_t>(phis) & amask) &&
                        !(reinterpret_cast<size_t>(phi) & amask) && !(reinterpret_cast<size_t>(acc) & amask) &&
                        !((size_t)ncell & 1);
    int last = -1;
    int ey0 = 0, ez0 = 0;
    unsigned ybase[4] = {0, 0, 0, 0}, zbase[4] = {0, 0, 0, 0};   // phis offsets of rows -1, 0, 1, 2 of the block
    unsigned prow = 0;
    for (FlatWalk it(f0, count, nbx); it.ok(); it.next()) {
        if (it.r != last) {
            last = it.r;
            const int by = it.r % nby, bz = it.r / nby;
            ey0 = 2 * by - g.acc_sh[1];
            ez0 = 2 * bz - g.acc_sh[2];
            // output cell e has phis index e + 1 on each axis; clamp into [0, W)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ybase[k] = sy * (unsigned)min(max(ey0 + k, 0), W1 - 1);
                zbase[k] = sz * (unsigned)min(max(ez0 + k, 0), W2 - 1);
            }
            if (carry) {
                // the odd level cell of the block's pair (2k+1) gives parent cell k
                const long long ky = ((g.start[1] + ey0 - 1) - 1) >> 1;
                const long long kz = ((g.start[2] + ez0 - 1) - 1) >> 1;
                prow = (unsigned)(ky - ps[1] + 1) * (unsigned)P0 + (unsigned)(kz - ps[2] + 1) * P01;
            }
        }
        const int ex0 = 2 * it.x - g.acc_sh[0];
        int xi[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) xi[k] = min(max(ex0 + k, 0), W0 - 1);
        // phis of the four centre rows at x indices ex0 .. ex0+3 (the x
        // neighbours and the centres e + 1 = ex0 + 1 + a): two pair loads when
        // the row is even-aligned and unclamped
        const bool vload = valign && ex0 >= 0 && ex0 + 3 <= W0 - 1 && !(ex0 & 1);
        T xr[2][2][4];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const unsigned row = zbase[1 + c] + ybase[1 + b];
                if (vload) {
                    const V2 u = *reinterpret_cast<const V2*>(phis + row + ex0);
                    const V2 v = *reinterpret_cast<const V2*>(phis + row + ex0 + 2);
                    xr[c][b][0] = u.x; xr[c][b][1] = u.y; xr[c][b][2] = v.x; xr[c][b][3] = v.y;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) xr[c][b][k] = phis[row + xi[k]];
                }
            }
        T out[2][2][2], q[2][2][2];
        unsigned pbase = 0;
        if (carry) {
            const long long kx = ((g.start[0] + ex0 - 1) - 1) >> 1;
            pbase = prow + (unsigned)(kx - ps[0] + 1);
            // the block's 8 parent cells: pbase .. pbase + 1 + P0 + P01
            if (!APM_IN_BOUNDS((long long)pbase + 1 + P0 + P01, pn, L.status)) continue;
        }
        // output cells: (ex0 + a, ey0 + b, ez0 + c); the pair a = 0, 1 is one
        // aligned pair store when both are inside and ex0 is even
        bool wr[2][2][2];
        unsigned o[2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int ey = ey0 + b, ez = ez0 + c;
                const bool yz = ey >= 0 && ey < E1 && ez >= 0 && ez < E2;
                wr[c][b][0] = yz && ex0 >= 0 && ex0 < E0;
                wr[c][b][1] = yz && ex0 + 1 < E0;
                o[c][b] = (unsigned)ex0 + (unsigned)E0 * ((unsigned)ey + (unsigned)E1 * (unsigned)ez);
            }
        const bool vpair = valign && !(ex0 & 1);
        auto put = [&](T* __restrict__ f, int c, int b, T v0, T v1) {
            if (vpair && wr[c][b][0] && wr[c][b][1]) {
                *reinterpret_cast<V2*>(f + o[c][b]) = mk2(v0, v1);
            } else {
                if (wr[c][b][0]) f[o[c][b]] = v0;
                if (wr[c][b][1]) f[o[c][b] + 1] = v1;
            }
        };
        // phi
        if (carry) {
            load_parent<T>(pphi, pbase, P0, P01, q);
            lerp_block<T>(q, out);
        }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                T v0 = xr[c][b][1], v1 = xr[c][b][2];
                if (carry) {
                    v0 += out[c][b][0];
                    v1 += out[c][b][1];
                }
                put(phi, c, b, v0, v1);
            }
        // acc_x: neighbours xr[.][.][0] and xr[.][.][3]
        {
            if (carry) {
                load_parent<T>(pacc, pbase, P0, P01, q);
                lerp_block<T>(q, out);
            }
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    T g0 = -(xr[c][b][2] - xr[c][b][0]) * inv2d;
                    T g1 = -(xr[c][b][3] - xr[c][b][1]) * inv2d;
                    if (carry) {
                        g0 += out[c][b][0];
                        g1 += out[c][b][1];
                    }
                    put(acc, c, b, g0, g1);
                }
        }
        // acc_y: rows ybase[0] and ybase[3]
        {
            if (carry) {
                load_parent<T>(pacc + pn, pbase, P0, P01, q);
                lerp_block<T>(q, out);
            }
            T gy[2][2][2];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const T lo = phis[zbase[1 + c] + ybase[0] + xi[1 + a]];
                    const T hi = phis[zbase[1 + c] + ybase[3] + xi[1 + a]];
                    gy[c][0][a] = -(xr[c][1][1 + a] - lo) * inv2d;
                    gy[c][1][a] = -(hi - xr[c][0][1 + a]) * inv2d;
                }
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    T v0 = gy[c][b][0], v1 = gy[c][b][1];
                    if (carry) {
                        v0 += out[c][b][0];
                        v1 += out[c][b][1];
                    }
                    put(acc + ncell, c, b, v0, v1);
                }
        }
        // acc_z: planes zbase[0] and zbase[3]
        {
            if (carry) {
                load_parent<T>(pacc + 2 * pn, pbase, P0, P01, q);
                lerp_block<T>(q, out);
            }
            T gz[2][2][2];
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const T lo = phis[zbase[0] + ybase[1 + b] + xi[1 + a]];
                    const T hi = phis[zbase[3] + ybase[1 + b] + xi[1 + a]];
                    gz[0][b][a] = -(xr[1][b][1 + a] - lo) * inv2d;
                    gz[1][b][a] = -(hi - xr[0][b][1 + a]) * inv2d;
                }
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    T v0 = gz[c][b][0], v1 = gz[c][b][1];
                    if (carry) {
                        v0 += out[c][b][0];
                        v1 += out[c][b][1];
                    }
                    put(acc + 2 * ncell, c, b, v0, v1);
                }
        }
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

// The 27 interpolation weights of a particle at fixed-point position X on a
// level with `fb` fraction bits.  FP64: the deposit's fixed-point weights
// exactly (outer products ((wx wy) wz) rounded on the scale 2^63, the centre one
// minus their sum).  FP32: the same TSC weights evaluated in FP32 from the
// offsets (t = f 2^-fb; (1-t)^2/2, 3/4 - (t-1/2)^2, t^2/2; products (wx wy) wz),
// within a few FP32 roundings of the fixed-point ones.
__device__ __forceinline__ void interp_weights(const long long X[3], int fb, double wq[3][3][3]) {
    unsigned long long w[3][3];
    for (int j = 0; j < 3; ++j) tsc_fixed(X[j], fb, w[j]);
    unsigned long long wsum = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == 1 && b == 1 && c == 1) continue;
                const unsigned long long q = wmul63(wmul63(w[0][a], w[1][b]), w[2][c]);
                wsum += q;
                wq[c][b][a] = __ull2double_rn(q) * 1.0842021724855044e-19;   // 2^-63
            }
    wq[1][1][1] = __ull2double_rn(kOne63 - wsum) * 1.0842021724855044e-19;
}
__device__ __forceinline__ void interp_weights(const long long X[3], int fb, float wq[3][3][3]) {
    float w[3][3];
    const float sc = __int_as_float((127 - fb) << 23);   // 2^-fb
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const long long i = X[j] >> fb;
        const float t = __uint2float_rn((unsigned)(X[j] - (i << fb))) * sc;   // offset < 2^fb <= 2^31
        const float u = 1.0f - t;
        w[j][0] = 0.5f * u * u;
        w[j][2] = 0.5f * t * t;
        w[j][1] = 0.75f - (t - 0.5f) * (t - 0.5f);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float wyz = w[1][b] * w[2][c];
#pragma unroll
            for (int a = 0; a < 3; ++a) wq[c][b][a] = w[0][a] * wyz;
        }
}

// TSC interpolation of the cell accelerations A (3 x (N+2)^3 of grid g, level L)
// at fixed-point position X; writes out[p], out[n + p], out[2n + p].
template <typename T>
__device__ __forceinline__ void interp_from(const LevelDev& L, const GridDev& g, const T* __restrict__ A,
                                            const long long X[3], long long p, long long n,
                                            T* __restrict__ out) {
    T wq[3][3][3];
    interp_weights(X, L.frac_bits, wq);
    const int E0 = g.N[0] + 2, E1 = g.N[1] + 2;
    const unsigned ncell = (unsigned)E0 * E1 * (g.N[2] + 2);
    const bool fold = g.mode == 1;
    int lc[3];
    for (int j = 0; j < 3; ++j) lc[j] = (int)((X[j] >> L.frac_bits) - g.start[j]);
    // the owner's interior holds the particle's cell (fold: the root's box)
    for (int j = 0; j < 3; ++j)
        if (!APM_IN_BOUNDS(fold ? min(max(lc[j], 0), g.N[j] - 1) : lc[j], g.N[j], L.status)) return;
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
                const T wt = wq[c][b][a];
                unsigned idx = (unsigned)(x + 1) + (unsigned)E0 * ((unsigned)(y + 1) + (unsigned)E1 * (unsigned)(z + 1));
                a0 += wt * A[idx];
                a1 += wt * A[ncell + idx];
                a2 += wt * A[2 * ncell + idx];
            }
        }
    }
    out[p] = a0;
    out[n + p] = a1;
    out[2 * n + p] = a2;
}

__device__ __forceinline__ void particle_position(const LevelDev& L, const Particles& P, long long p,
                                                  double half_dt, long long X[3]) {
    X[0] = fixed_position(drift_raw(P.x[p], P.vx[p], half_dt), L);
    X[1] = fixed_position(drift_raw(P.y[p], P.vy[p], half_dt), L);
    X[2] = fixed_position(drift_raw(P.z[p], P.vz[p], half_dt), L);
}

// One level: the particles owned by a grid of L and by no grid of the finer
// level F (the finest grid holding a particle supplies its acceleration).
template <typename T>
__global__ void __launch_bounds__(256) k_interp(LevelDev L, LevelDev F, int has_finer, Particles P,
                                                double half_dt, const void* const* __restrict__ acc_p,
                                                T* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const long long p = P.at(i);
    long long X[3];
    particle_position(L, P, p, half_dt, X);
    long long ic[3];
    for (int j = 0; j < 3; ++j) ic[j] = X[j] >> L.frac_bits;
    int gi = find_owner(L, ic);
    if (gi < 0) return;
    if (has_finer) {
        long long fc[3];
        for (int j = 0; j < 3; ++j) fc[j] = X[j] >> F.frac_bits;
        if (find_owner(F, fc) >= 0) return;
    }
    interp_from<T>(L, L.g[gi], reinterpret_cast<const T*>(acc_p[gi]), X, p, P.n, out);
}

// Every level in one pass: each particle's position is converted once and its
// owner searched from the root down (a finer owner lies inside a coarser one);
// the finest owner supplies the acceleration.  accs[l]: the acceleration
// pointer table of level l.
// CTA size and minimum resident CTAs per SM of the all-level interpolation
#ifndef APM_INT_THREADS
#define APM_INT_THREADS 128
#endif
#ifndef APM_INT_MIN_CTAS
#define APM_INT_MIN_CTAS 8
#endif
constexpr int kIntThreads = APM_INT_THREADS;

template <typename T>
__global__ void __launch_bounds__(kIntThreads, APM_INT_MIN_CTAS) k_interp_levels(const LevelDev* __restrict__ levels, int nl, Particles P,
                                                       double half_dt, const void* const* const* __restrict__ accs,
                                                       T* __restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const long long p = P.at(i);
    long long X[3];
    particle_position(levels[0], P, p, half_dt, X);
    int own_l = -1, own_g = -1;
    for (int l = 0; l < nl; ++l) {
        long long ic[3];
        for (int j = 0; j < 3; ++j) ic[j] = X[j] >> levels[l].frac_bits;
        const int gi = find_owner(levels[l], ic);
        if (gi < 0) break;
        own_l = l;
        own_g = gi;
    }
    if (own_l < 0) return;
    const LevelDev& L = levels[own_l];
    interp_from<T>(L, L.g[own_g], reinterpret_cast<const T*>(accs[own_l][own_g]), X, p, P.n, out);
}

// Four-point and spectral gradients (Sec. 2.2; apm_gradient), on the 2x2x2
// blocks of k_accel (same work list, same parent interpolation):
//   phi(c)   = phis(c) + I(parent phi)(c)
//   acc_j(c) = A_j(c) + I(parent acc_j)(c),        c in [-1, N]^3, with
//   A_j = -(8 (phis(c+e_j) - phis(c-e_j)) - (phis(c+2e_j) - phis(c-2e_j))) / (12 delta)
//         (four-point; phis spans [-3, N+3)), or the solve's spectral component
//         j + 1 (phis: four windows of [-2, N+2)).
// Output cell e (index 0..E-1) is level cell e - 1 and phis cell e - 1 + h.
template <typename T, int GRAD>
__global__ void __launch_bounds__(kAccThreads, AccMinCtas<T>::value) k_accel_var(
    LevelDev L, const GridDev* __restrict__ pgrids, const void* const* __restrict__ phis_p,
    const void* const* __restrict__ pphi_p, const void* const* __restrict__ pacc_p,
    void* const* __restrict__ phi_p, void* const* __restrict__ acc_p, const Chunk* __restrict__ chunks) {
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = L.g[ch.grid];
    const int E0 = g.N[0] + 2, E1 = g.N[1] + 2, E2 = g.N[2] + 2;
    const unsigned ncell = (unsigned)E0 * E1 * E2;
    const int h = g.h;
    const unsigned W0 = g.W[0], W01 = (unsigned)g.W[0] * g.W[1];
    const unsigned nw = W01 * (unsigned)g.W[2];
    const int nbx = g.acc_nb[0], nby = g.acc_nb[1];
    const int nbrows = nby * g.acc_nb[2];
    const T* __restrict__ phis = reinterpret_cast<const T*>(phis_p[ch.grid]);
    T* __restrict__ phi = reinterpret_cast<T*>(phi_p[ch.grid]);
    T* __restrict__ acc = reinterpret_cast<T*>(acc_p[ch.grid]);
    const bool carry = pphi_p != nullptr && g.parent >= 0;
    const T* __restrict__ pphi = carry ? reinterpret_cast<const T*>(pphi_p[g.parent]) : nullptr;
    const T* __restrict__ pacc = carry ? reinterpret_cast<const T*>(pacc_p[g.parent]) : nullptr;
    int P0 = 0;
    unsigned P01 = 0, pn = 0;
    long long ps[3] = {0, 0, 0};
    if (carry) {
        const GridDev& p = pgrids[g.parent];
        P0 = p.N[0] + 2;
        P01 = (unsigned)P0 * (p.N[1] + 2);
        pn = P01 * (p.N[2] + 2);
        ps[0] = p.start[0]; ps[1] = p.start[1]; ps[2] = p.start[2];
    }
    const T inv12d = (T)g.inv12d;
    const unsigned st[3] = {1u, W0, W01};
    // two-element accesses need even row lengths and pointers aligned to two elements
    using V2 = typename Cplx<T>::type;
    const size_t amask = 2 * sizeof(T) - 1;
    const bool vout = !(E0 & 1) && !(ncell & 1) && !(reinterpret_cast<size_t>(phi) & amask) &&
                      !(reinterpret_cast<size_t>(acc) & amask);
    const bool vin = !(W0 & 1) && !(W01 & 1) && !(nw & 1) && !(reinterpret_cast<size_t>(phis) & amask);
    const long long nblocks = (long long)nbx * nbrows;
    const long long f0 = (long long)ch.tile * kAccBlocksPerCta;
    const int count = (int)min((long long)kAccBlocksPerCta, nblocks - f0);
    int last = -1;
    int ey0 = 0, ez0 = 0;
    unsigned prow = 0;
    for (FlatWalk it(f0, count, nbx); it.ok(); it.next()) {
        if (it.r != last) {
            last = it.r;
            const int by = it.r % nby, bz = it.r / nby;
            ey0 = 2 * by - g.acc_sh[1];
            ez0 = 2 * bz - g.acc_sh[2];
            if (carry) {
                const long long ky = ((g.start[1] + ey0 - 1) - 1) >> 1;
                const long long kz = ((g.start[2] + ez0 - 1) - 1) >> 1;
                prow = (unsigned)(ky - ps[1] + 1) * (unsigned)P0 + (unsigned)(kz - ps[2] + 1) * P01;
            }
        }
        const int ex0 = 2 * it.x - g.acc_sh[0];
        unsigned pbase = 0;
        if (carry) {
            const long long kx = ((g.start[0] + ex0 - 1) - 1) >> 1;
            pbase = prow + (unsigned)(kx - ps[0] + 1);
            if (!APM_IN_BOUNDS((long long)pbase + 1 + P0 + P01, pn, L.status)) continue;
        }
        bool wr[2][2][2];
        unsigned o[2][2][2], c0[2][2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int ex = ex0 + a, ey = ey0 + b, ez = ez0 + c;
                    wr[c][b][a] = ex >= 0 && ex < E0 && ey >= 0 && ey < E1 && ez >= 0 && ez < E2;
                    o[c][b][a] = (unsigned)ex + (unsigned)E0 * ((unsigned)ey + (unsigned)E1 * (unsigned)ez);
                    c0[c][b][a] = (unsigned)(ex - 1 + h) + W0 * (unsigned)(ey - 1 + h) + W01 * (unsigned)(ez - 1 + h);
                }
        // a row pair (a = 0, 1) with both cells written moves as two-element
        // loads and stores where aligned; other pairs cell by cell
        const bool pst = vout && !(ex0 & 1);               // o[.][.][0] even
        const bool pld = vin && !(c0[0][0][0] & 1);        // c0[.][.][0] even (W0, W01 even)
        T out[2][2][2], q[2][2][2];
        if (carry) {
            load_parent<T>(pphi, pbase, P0, P01, q);
            lerp_block<T>(q, out);
        }
        auto put = [&](T* __restrict__ f, unsigned i, int c, int b, T v0, T v1) {
            if (pst && wr[c][b][0] && wr[c][b][1]) {
                *reinterpret_cast<V2*>(f + i) = mk2(v0, v1);
            } else {
                if (wr[c][b][0]) f[i] = v0;
                if (wr[c][b][1]) f[i + 1] = v1;
            }
        };
        auto ld2 = [&](const T* __restrict__ f, unsigned i, T& v0, T& v1) {
            if (pld) {
                const V2 u = *reinterpret_cast<const V2*>(f + i);
                v0 = u.x;
                v1 = u.y;
            } else {
                v0 = f[i];
                v1 = f[i + 1];
            }
        };
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const unsigned ci = c0[c][b][0];
                T v0 = 0, v1 = 0;
                if (wr[c][b][0] && wr[c][b][1]) {
                    ld2(phis, ci, v0, v1);
                } else {
                    if (wr[c][b][0]) v0 = phis[ci];
                    if (wr[c][b][1]) v1 = phis[ci + 1];
                }
                if (carry) {
                    v0 += out[c][b][0];
                    v1 += out[c][b][1];
                }
                put(phi, o[c][b][0], c, b, v0, v1);
            }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (carry) {
                load_parent<T>(pacc + j * pn, pbase, P0, P01, q);
                lerp_block<T>(q, out);
            }
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const unsigned ci = c0[c][b][0];
                    T v[2] = {0, 0};
                    if (wr[c][b][0] && wr[c][b][1]) {
                        if constexpr (GRAD == APM_GRAD_FD4) {
                            if (j == 0) {   // x: cells ci-2 .. ci+3
                                T m2, m1, p0, p1, p2, p3;
                                ld2(phis, ci - 2, m2, m1);
                                ld2(phis, ci, p0, p1);
                                ld2(phis, ci + 2, p2, p3);
                                v[0] = -((T)8 * (p1 - m1) - (p2 - m2)) * inv12d;
                                v[1] = -((T)8 * (p2 - p0) - (p3 - m1)) * inv12d;
                            } else {
                                T a1[2], b1[2], a2[2], b2[2];
                                ld2(phis, ci + st[j], a1[0], a1[1]);
                                ld2(phis, ci - st[j], b1[0], b1[1]);
                                ld2(phis, ci + 2 * st[j], a2[0], a2[1]);
                                ld2(phis, ci - 2 * st[j], b2[0], b2[1]);
#pragma unroll
                                for (int a = 0; a < 2; ++a)
                                    v[a] = -((T)8 * (a1[a] - b1[a]) - (a2[a] - b2[a])) * inv12d;
                            }
                        } else {
                            ld2(phis, (j + 1) * nw + ci, v[0], v[1]);
                        }
                    } else {
#pragma unroll
                        for (int a = 0; a < 2; ++a) {
                            if (!wr[c][b][a]) continue;
                            const unsigned cc = ci + a;
                            if constexpr (GRAD == APM_GRAD_FD4) {
                                const T d1 = phis[cc + st[j]] - phis[cc - st[j]];
                                const T d2 = phis[cc + 2 * st[j]] - phis[cc - 2 * st[j]];
                                v[a] = -((T)8 * d1 - d2) * inv12d;
                            } else {
                                v[a] = phis[(j + 1) * nw + cc];
                            }
                        }
                    }
                    if (carry) {
                        v[0] += out[c][b][0];
                        v[1] += out[c][b][1];
                    }
                    put(acc + j * ncell, o[c][b][0], c, b, v[0], v[1]);
                }
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_accel(const LevelDev& L, const GridDev* parent_grids, const void* const* phis,
                         const void* const* pphi, const void* const* pacc, void* const* phi,
                         void* const* acc, const Chunk* chunks, int n_chunks,
                         cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    k_accel<T><<<n_chunks, kAccThreads, 0, s>>>(L, parent_grids, phis, pphi, pacc, phi, acc, chunks);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_accel_var(const LevelDev& L, const GridDev* parent_grids, const void* const* phis,
                               const void* const* pphi, const void* const* pacc, void* const* phi,
                               void* const* acc, const Chunk* chunks, int n_chunks, int grad,
                               cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    if (grad == APM_GRAD_FD4)
        k_accel_var<T, APM_GRAD_FD4><<<n_chunks, kAccThreads, 0, s>>>(L, parent_grids, phis, pphi, pacc, phi, acc,
                                                                      chunks);
    else
        k_accel_var<T, APM_GRAD_SPECTRAL><<<n_chunks, kAccThreads, 0, s>>>(L, parent_grids, phis, pphi, pacc, phi,
                                                                           acc, chunks);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interp(const LevelDev& L, const LevelDev* finer, const Particles& P,
                          double half_dt, const void* const* acc, void* out, cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((P.n + 255) / 256);
    LevelDev F = finer ? *finer : L;
    k_interp<T><<<blocks, 256, 0, s>>>(L, F, finer ? 1 : 0, P, half_dt, acc, reinterpret_cast<T*>(out));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interp_levels(const LevelDev* levels, int nl, const Particles& P, double half_dt,
                                 const void* const* const* accs, void* out, cudaStream_t s) {
    if (P.n <= 0 || nl <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((P.n + kIntThreads - 1) / kIntThreads);
    k_interp_levels<T><<<blocks, kIntThreads, 0, s>>>(levels, nl, P, half_dt, accs, reinterpret_cast<T*>(out));
    return cudaGetLastError();
}

template cudaError_t launch_accel<float>(const LevelDev&, const GridDev*, const void* const*,
                                         const void* const*, const void* const*, void* const*,
                                         void* const*, const Chunk*, int, cudaStream_t);
template cudaError_t launch_accel<double>(const LevelDev&, const GridDev*, const void* const*,
                                          const void* const*, const void* const*, void* const*,
                                          void* const*, const Chunk*, int, cudaStream_t);
template cudaError_t launch_accel_var<float>(const LevelDev&, const GridDev*, const void* const*,
                                               const void* const*, const void* const*, void* const*,
                                               void* const*, const Chunk*, int, int, cudaStream_t);
template cudaError_t launch_accel_var<double>(const LevelDev&, const GridDev*, const void* const*,
                                                const void* const*, const void* const*, void* const*,
                                                void* const*, const Chunk*, int, int, cudaStream_t);
template cudaError_t launch_interp<float>(const LevelDev&, const LevelDev*, const Particles&, double,
                                          const void* const*, void*, cudaStream_t);
template cudaError_t launch_interp<double>(const LevelDev&, const LevelDev*, const Particles&, double,
                                           const void* const*, void*, cudaStream_t);
template cudaError_t launch_interp_levels<float>(const LevelDev*, int, const Particles&, double,
                                                 const void* const* const*, void*, cudaStream_t);
template cudaError_t launch_interp_levels<double>(const LevelDev*, int, const Particles&, double,
                                                  const void* const* const*, void*, cudaStream_t);

}  // namespace apm

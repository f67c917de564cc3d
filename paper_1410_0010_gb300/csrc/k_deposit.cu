// k_deposit.cu -- gravitating-mass field (GMF) of every grid of a level (Sec. 2):
// baryons (interior gas, parent gas copied onto the border) initialise every
// cell, then each particle, drifted half a timestep, adds its 27 TSC charges
// in 64-bit fixed point with integer atomics.  Integer addition is exact and
// associative, so the field is bit-identical for any particle order and any
// atomic interleaving.  Every floating-point step uses explicitly rounded
// intrinsics (no contraction), so the charges equal a plain IEEE evaluation.
#include "apm_internal.cuh"

namespace apm {
namespace {

__device__ __forceinline__ long long floor_div(long long a, long long b) {
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// One CTA per batch of `rows` GMF rows (a row: G0 cells along x at fixed y, z).
__global__ void __launch_bounds__(256) k_gas_init(LevelDev L, const GridDev* __restrict__ pgrids,
                           const double* const* __restrict__ gas,
                           const double* const* __restrict__ pgas, int64_t* const* __restrict__ gmf,
                           const Chunk* __restrict__ chunks, int rows_per_cta, int F, int refine) {
    const Chunk c = chunks[blockIdx.x];
    const GridDev& g = L.g[c.grid];
    const int G0 = g.G[0], G1 = g.G[1];
    const int nrows = G1 * g.G[2];
    const double scale = ldexp(1.0, F);
    const double vol = __dmul_rn(__dmul_rn(g.delta, g.delta), g.delta);
    const double* own = gas ? gas[c.grid] : nullptr;
    const double* par = (pgas && g.parent >= 0) ? pgas[g.parent] : nullptr;
    int64_t* __restrict__ out = gmf[c.grid];
    const int B = (G0 - g.N[0]) / 2;
    const int r0 = c.tile * g.rows_gas;
    const int r1 = min(nrows, r0 + g.rows_gas);
    for (int r = r0; r < r1; ++r) {
        int64_t* row = out + (long long)r * G0;
        if (!own && !par) {
            for (int x = threadIdx.x; x < G0; x += blockDim.x) row[x] = 0;
            continue;
        }
        const int y = r % G1, z = r / G1;
        const int cy = y - B, cz = z - B;
        const bool yz_in = cy >= 0 && cy < g.N[1] && cz >= 0 && cz < g.N[2];
        for (int x = threadIdx.x; x < G0; x += blockDim.x) {
            const int cx = x - B;
            double rho = 0.0;
            if (yz_in && cx >= 0 && cx < g.N[0]) {
                if (own) rho = own[cx + (long long)g.N[0] * (cy + (long long)g.N[1] * cz)];
            } else if (par) {
                const GridDev& p = pgrids[g.parent];
                long long px = floor_div(g.start[0] + cx, refine) - p.start[0];
                long long py = floor_div(g.start[1] + cy, refine) - p.start[1];
                long long pz = floor_div(g.start[2] + cz, refine) - p.start[2];
                rho = par[px + (long long)p.N[0] * (py + (long long)p.N[1] * pz)];
            }
            row[x] = __double2ll_rn(__dmul_rn(__dmul_rn(rho, vol), scale));
        }
    }
}

// x' = x + v half_dt; on a periodic domain x' - box floor(x'/box), which is x'
// itself (bit for bit) when x' is already inside [0, box)
__device__ __forceinline__ double drift(double x, double v, double half_dt, double box,
                                        int periodic) {
    double xd = __dadd_rn(x, __dmul_rn(v, half_dt));
    if (periodic && !(xd >= 0.0 && xd < box))
        xd = __dsub_rn(xd, __dmul_rn(box, floor(__ddiv_rn(xd, box))));
    return xd;
}

// adds the 27 charges q (z-major: q[c][b][a]) to one GMF box
__device__ __forceinline__ void scatter(const GridDev& g, int64_t* __restrict__ out,
                                        const long long ic[3], const long long q[3][3][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        long long z = ic[2] + c - 1 - g.lo[2];
        if (g.mode == 1) z = z < 0 ? 0 : (z >= g.G[2] ? g.G[2] - 1 : z);
        else if (g.mode == 2) { z %= g.G[2]; if (z < 0) z += g.G[2]; }
        else if (z < 0 || z >= g.G[2]) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            long long y = ic[1] + b - 1 - g.lo[1];
            if (g.mode == 1) y = y < 0 ? 0 : (y >= g.G[1] ? g.G[1] - 1 : y);
            else if (g.mode == 2) { y %= g.G[1]; if (y < 0) y += g.G[1]; }
            else if (y < 0 || y >= g.G[1]) continue;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                long long x = ic[0] + a - 1 - g.lo[0];
                if (g.mode == 1) x = x < 0 ? 0 : (x >= g.G[0] ? g.G[0] - 1 : x);
                else if (g.mode == 2) { x %= g.G[0]; if (x < 0) x += g.G[0]; }
                else if (x < 0 || x >= g.G[0]) continue;
                long long q0 = q[c][b][a];
                if (q0 != 0)
                    atomicAdd(reinterpret_cast<unsigned long long*>(
                                  out + (x + (long long)g.G[0] * (y + (long long)g.G[1] * z))),
                              (unsigned long long)q0);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_deposit(LevelDev L, Particles P, double half_dt,
                                                 double box, int periodic, int F,
                                                 int64_t* const* __restrict__ gmf,
                                                 unsigned* __restrict__ status) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P.n) return;
    const double x = P.x[p], y = P.y[p], z = P.z[p];
    const double vx = P.vx[p], vy = P.vy[p], vz = P.vz[p];
    if (!L.is_root && L.cull_fp32) {
        // FP32 estimate of the particle's tile (error far below the 4-cell tile):
        // particles with no occupied tile nearby touch no GMF box of this level
        const TileMap& m = L.map;
        const float hf = (float)half_dt, inv = (float)L.inv_delta;
        const float px[3] = {((float)x + (float)vx * hf) * inv, ((float)y + (float)vy * hf) * inv,
                             ((float)z + (float)vz * hf) * inv};
        long long t[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float rel = floorf(px[j]) - (float)m.lo[j];
            if (!(rel > -4.0f)) return;
            t[j] = rel < 0.0f ? 0 : ((long long)rel >> m.shift);
            if (t[j] >= m.nt[j]) {
                if (t[j] > m.nt[j]) return;
                t[j] = m.nt[j] - 1;
            }
        }
        if (!m.occ[t[0] + (long long)m.nt[0] * (t[1] + (long long)m.nt[1] * t[2])]) return;
    }
    // fixed-point position and weights (the same for every level)
    long long ic[3];
    unsigned long long w[3][3];
    const int PB = L.frac_bits;
    const double xd[3] = {drift(x, vx, half_dt, box, periodic), drift(y, vy, half_dt, box, periodic),
                          drift(z, vz, half_dt, box, periodic)};
#pragma unroll
    for (int j = 0; j < 3; ++j) ic[j] = tsc_fixed(fixed_position(xd[j], L), PB, w[j]);

    // candidate grids
    int e0 = 0, e1 = 1;
    if (!L.is_root) {
        const TileMap& m = L.map;
        long long t[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            long long rel = ic[j] - m.lo[j];
            if (rel < 0) return;
            t[j] = rel >> m.shift;
            if (t[j] >= m.nt[j]) return;
        }
        long long tile = t[0] + (long long)m.nt[0] * (t[1] + (long long)m.nt[1] * t[2]);
        e0 = m.dep_off[tile];
        e1 = m.dep_off[tile + 1];
        if (e0 == e1) return;
    }

    const double mq = __dmul_rn(P.m[p], ldexp(1.0, F));
    if (!(fabs(mq) < 4611686018427387904.0)) {   // 2^62
        atomicOr(status, kStOverflow);
        return;
    }
    const long long M = __double2ll_rn(mq);
    const unsigned long long aM = (unsigned long long)(M < 0 ? -M : M);
    // charges (|M| w + 2^62) >> 63 of the 26 outer cells, w = ((wx wy) wz) each
    // product rounded half up; the centre takes M minus the others
    long long q[3][3][3];
    long long others = 0;
    unsigned long long wxy[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) wxy[b][a] = wmul63(w[0][a], w[1][b]);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == 1 && b == 1 && c == 1) continue;
                long long v = (long long)wmul63(aM, wmul63(wxy[b][a], w[2][c]));
                q[c][b][a] = M < 0 ? -v : v;
                others += q[c][b][a];
            }
    q[1][1][1] = M - others;

    for (int e = e0; e < e1; ++e) {
        int gi = L.is_root ? 0 : L.map.dep_list[e];
        const GridDev& g = L.g[gi];
        if (g.mode == 1) {
            for (int j = 0; j < 3; ++j)
                if (!(xd[j] >= 0.0 && xd[j] < box)) atomicOr(status, kStOutOfBox);
        }
        scatter(g, gmf[gi], ic, q);
    }
}

}  // namespace

cudaError_t launch_gas_init(const LevelDev& L, const GridDev* parent_grids,
                            const double* const* gas, const double* const* pgas,
                            int64_t* const* gmf, const Chunk* chunks, int n_chunks, int rows_per_cta,
                            int F, cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    k_gas_init<<<n_chunks, 256, 0, s>>>(L, parent_grids, gas, pgas, gmf, chunks, rows_per_cta, F,
                                         L.refine);
    return cudaGetLastError();
}

cudaError_t launch_deposit(const LevelDev& L, const Particles& P, double half_dt, double box,
                           int periodic, int F, int64_t* const* gmf, unsigned* status,
                           cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((P.n + 255) / 256);
    k_deposit<<<blocks, 256, 0, s>>>(L, P, half_dt, box, periodic, F, gmf, status);
    return cudaGetLastError();
}

}  // namespace apm

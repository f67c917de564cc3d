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

__global__ void k_gas_init(LevelDev L, const GridDev* __restrict__ pgrids,
                           const double* const* __restrict__ gas,
                           const double* const* __restrict__ pgas, int64_t* const* __restrict__ gmf,
                           const Chunk* __restrict__ chunks, int chunk_cells, int F, int refine) {
    const Chunk c = chunks[blockIdx.x];
    const GridDev& g = L.g[c.grid];
    const double scale = ldexp(1.0, F);
    const double vol = __dmul_rn(__dmul_rn(g.delta, g.delta), g.delta);
    const double* own = gas ? gas[c.grid] : nullptr;
    const double* par = (pgas && g.parent >= 0) ? pgas[g.parent] : nullptr;
    int64_t* out = gmf[c.grid];
    const int B = (g.G[0] - g.N[0]) / 2;
    long long cell0 = (long long)c.tile * chunk_cells;
    for (int t = threadIdx.x; t < chunk_cells; t += blockDim.x) {
        long long cell = cell0 + t;
        if (cell >= g.cells_gmf) break;
        int x = (int)(cell % g.G[0]);
        long long r = cell / g.G[0];
        int y = (int)(r % g.G[1]);
        int z = (int)(r / g.G[1]);
        int cx = x - B, cy = y - B, cz = z - B;
        double rho = 0.0;
        if (cx >= 0 && cx < g.N[0] && cy >= 0 && cy < g.N[1] && cz >= 0 && cz < g.N[2]) {
            if (own) rho = own[cx + (long long)g.N[0] * (cy + (long long)g.N[1] * cz)];
        } else if (par) {
            const GridDev& p = pgrids[g.parent];
            long long px = floor_div(g.start[0] + cx, refine) - p.start[0];
            long long py = floor_div(g.start[1] + cy, refine) - p.start[1];
            long long pz = floor_div(g.start[2] + cz, refine) - p.start[2];
            rho = par[px + (long long)p.N[0] * (py + (long long)p.N[1] * pz)];
        }
        out[cell] = __double2ll_rn(__dmul_rn(__dmul_rn(rho, vol), scale));
    }
}

struct Tsc {
    long long i[3];   // cell holding the particle, per axis
    double w[3][3];   // weights of cells i-1, i, i+1
};

// u = x / delta; when delta is a power of two the product with 1/delta is the
// same number (exact scaling) and avoids the FP64 division
__device__ __forceinline__ double to_cells(double xd, const LevelDev& L) {
    return L.delta_pow2 ? __dmul_rn(xd, L.inv_delta) : __ddiv_rn(xd, L.delta);
}

__device__ __forceinline__ void tsc_axis(double u, long long& i, double w[3]) {
    double fi = floor(u);
    double d = __dsub_rn(__dsub_rn(u, fi), 0.5);
    double a = __dsub_rn(0.5, d);
    double b = __dadd_rn(0.5, d);
    w[0] = __dmul_rn(0.5, __dmul_rn(a, a));
    w[1] = __dsub_rn(0.75, __dmul_rn(d, d));
    w[2] = __dmul_rn(0.5, __dmul_rn(b, b));
    i = (long long)fi;
}

__device__ __forceinline__ double drift(double x, double v, double half_dt, double box,
                                        int periodic) {
    double xd = __dadd_rn(x, __dmul_rn(v, half_dt));
    if (periodic) xd = __dsub_rn(xd, __dmul_rn(box, floor(__ddiv_rn(xd, box))));
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
    long long ic[3];
    double w[3][3];
    tsc_axis(to_cells(drift(x, vx, half_dt, box, periodic), L), ic[0], w[0]);
    tsc_axis(to_cells(drift(y, vy, half_dt, box, periodic), L), ic[1], w[1]);
    tsc_axis(to_cells(drift(z, vz, half_dt, box, periodic), L), ic[2], w[2]);

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

    const double scale = ldexp(1.0, F);
    const double mass = P.m[p];
    const double mq = __dmul_rn(mass, scale);
    if (!(fabs(mq) < 4611686018427387904.0)) {   // 2^62
        atomicOr(status, kStOverflow);
        return;
    }
    long long q[3][3][3];
    long long others = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == 1 && b == 1 && c == 1) continue;
                double wt = __dmul_rn(__dmul_rn(w[0][a], w[1][b]), w[2][c]);
                q[c][b][a] = __double2ll_rn(__dmul_rn(__dmul_rn(mass, wt), scale));
                others += q[c][b][a];
            }
    q[1][1][1] = __double2ll_rn(mq) - others;

    for (int e = e0; e < e1; ++e) {
        int gi = L.is_root ? 0 : L.map.dep_list[e];
        const GridDev& g = L.g[gi];
        if (g.mode == 1) {
            for (int j = 0; j < 3; ++j)
                if (ic[j] < 0 || ic[j] >= g.G[j]) atomicOr(status, kStOutOfBox);
        }
        scatter(g, gmf[gi], ic, q);
    }
}

}  // namespace

cudaError_t launch_gas_init(const LevelDev& L, const GridDev* parent_grids,
                            const double* const* gas, const double* const* pgas,
                            int64_t* const* gmf, const Chunk* chunks, int n_chunks, int chunk_cells,
                            int F, cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    k_gas_init<<<n_chunks, 256, 0, s>>>(L, parent_grids, gas, pgas, gmf, chunks, chunk_cells, F,
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

// k_deposit.cu -- gravitating-mass field (GMF) of every grid of a level (Sec. 2):
// baryons (interior gas, parent gas copied onto the border) initialise every
// cell, then each particle, drifted half a timestep, adds its 27 TSC charges
// in 64-bit fixed point with integer atomics.  Integer addition is exact and
// associative, so the field is bit-identical for any particle order and any
// atomic interleaving.  Every floating-point step uses explicitly rounded
// intrinsics (no contraction), so the charges equal a plain IEEE evaluation.
#include <climits>

#include "apm_internal.cuh"

namespace apm {
namespace {


// no baryons: the CTA's rows are one flat range of n zeros, written as
// 16-byte stores when the range starts 16-byte aligned
__device__ __noinline__ void zero_range(int64_t* __restrict__ z, long long n) {
    long long i0 = 0;
    if ((reinterpret_cast<size_t>(z) & 15) == 0) {
        longlong2* __restrict__ z2 = reinterpret_cast<longlong2*>(z);
        for (long long i = threadIdx.x; i < n / 2; i += blockDim.x) z2[i] = make_longlong2(0, 0);
        i0 = n & ~1LL;
    }
    for (long long i = i0 + threadIdx.x; i < n; i += blockDim.x) z[i] = 0;
}

// One CTA per batch of `rows` GMF rows (a row: G0 cells along x at fixed y, z).
__global__ void __launch_bounds__(256) k_gas_init(LevelDev L, const GridDev* __restrict__ pgrids,
                           const double* const* __restrict__ gas,
                           const double* const* __restrict__ pgas, int64_t* const* __restrict__ gmf,
                           const Chunk* __restrict__ chunks, int F) {
    const Chunk c = chunks[blockIdx.x];
    const GridDev& g = L.g[c.grid];
    const int G0 = g.G[0], G1 = g.G[1];
    const int nrows = G1 * g.G[2];
    const double scale = ldexp(1.0, F);
    const double vol = __dmul_rn(__dmul_rn(g.delta, g.delta), g.delta);
    // when delta is a power of two, 2^e, the two products are exact exponent
    // shifts and rint((rho delta^3) 2^F) = rint(rho 2^(F + 3e)), which
    // scaled_rint computes with integer operations (the FP64 products remain
    // for other cell sizes and for values scaled_rint cannot hold)
    const unsigned long long db = (unsigned long long)__double_as_longlong(g.delta);
    const int de = (int)((db >> 52) & 0x7FF);
    const bool pow2 = (db & 0xFFFFFFFFFFFFFULL) == 0 && de > 0 && de < 0x7FF;
    const int K = F + 3 * (de - 1023);
    const double* own = gas ? gas[c.grid] : nullptr;
    const double* par = (pgas && g.parent >= 0) ? pgas[g.parent] : nullptr;
    int64_t* __restrict__ out = gmf[c.grid];
    const int B = (G0 - g.N[0]) / 2;
    const int r0 = c.tile * g.rows_gas;
    const int r1 = min(nrows, r0 + g.rows_gas);
    const GridDev* p = par ? &pgrids[g.parent] : nullptr;
    if (!own && !par) {
        zero_range(out + (long long)r0 * G0, (long long)(r1 - r0) * G0);
        return;
    }
    int last = -1, cy = 0, cz = 0;
    bool yz_in = false;
    for (RowWalk it(r0, G0); it.r < r1; it.next()) {
        const int r = it.r, x = it.x;
        int64_t* row = out + (long long)r * G0;
        if (r != last) {
            last = r;
            cy = r % G1 - B;
            cz = r / G1 - B;
            yz_in = cy >= 0 && cy < g.N[1] && cz >= 0 && cz < g.N[2];
        }
        const int cx = x - B;
        double rho = 0.0;
        if (yz_in && cx >= 0 && cx < g.N[0]) {
            if (own) rho = own[cx + (long long)g.N[0] * (cy + (long long)g.N[1] * cz)];
        } else if (par) {
            // parent cell floor(c / 2): the refinement factor is 2 (checked on the host);
            // past an isolated root's faces (the only border cells with no parent
            // cell, checked on the host) there are no baryons
            long long px = ((g.start[0] + cx) >> 1) - p->start[0];
            long long py = ((g.start[1] + cy) >> 1) - p->start[1];
            long long pz = ((g.start[2] + cz) >> 1) - p->start[2];
            if (px >= 0 && px < p->N[0] && py >= 0 && py < p->N[1] && pz >= 0 && pz < p->N[2])
                rho = par[px + (long long)p->N[0] * (py + (long long)p->N[1] * pz)];
        }
        if (APM_IN_BOUNDS((long long)r * G0 + x, g.cells_gmf, L.status)) {
            bool ok = false;
            long long v = pow2 ? scaled_rint(rho, K, ok) : 0;
            if (!ok) v = __double2ll_rn(__dmul_rn(__dmul_rn(rho, vol), scale));
            row[x] = v;
        }
    }
}


// GMF-local index of one cloud cell per axis under the grid's edge rule
// (mode 0 drop: -1 when outside, 1 fold, 2 wrap)
// (on the periodic root the centre cell is in [0, G), so v is in [-1, G])
__device__ __forceinline__ int edge_rule(long long v, int G, int mode) {
    if (mode == 1) return v < 0 ? 0 : (v >= G ? G - 1 : (int)v);
    if (mode == 2) return (int)(v < 0 ? v + G : (v >= G ? v - G : v));
    return (v < 0 || v >= G) ? -1 : (int)v;
}

// out[idx] += q as a fire-and-forget reduction (red: no value comes back, so
// the issuing warp never waits on it); two's-complement addition mod 2^64 is
// the same for signed and unsigned operands
__device__ __forceinline__ void add_charge(int64_t* __restrict__ out, unsigned idx, long long q) {
    if (q != 0)
        asm volatile("red.global.add.u64 [%0], %1;" ::"l"(out + idx), "l"((unsigned long long)q));
}

// ---- the deposit of particles in bin order: per-CTA tiles in shared memory ----
// With the particles sorted by bins of 2^s root cells (apm_order_particles,
// x fastest), a CTA's particles lie in one bin or in two x-neighbours, and
// their clouds overlap.  For each level whose tile fits kTileCells, the CTA
// keeps the charges that fall into one grid's box around its first
// candidate particle's bin (that bin and the next along x, with one cell of
// halo) in shared memory: each 64-bit sum is two 32-bit words, added with
// native 32-bit atomics, the low word's carry going to the high word, so the
// sum is exact modulo 2^64.  Charges outside the box, or to another grid, go
// straight to L2.  After a barrier the CTA sends one reduction per nonzero
// cell.  Integer sums do not depend on the order: the field is bit-identical
// to the direct deposit's.
constexpr int kTileCells = 2304;    // 9 KB of low words and 9 KB of high words
constexpr int kMaxTileLevels = 4;
struct DepTile {
    int gi;          // the grid (index on the level), < 0: no tile
    int o[3];        // box origin in the grid's GMF cells
    int n[3];        // box extents
    int base;        // first cell in the words
};
struct TileSet {
    DepTile* t;      // per tile slot
    unsigned* lo;
    unsigned* hi;
};

// v into slot `slot`'s tile when grid gi's cell (cx, cy, cz) lies in it
__device__ __forceinline__ bool tile_add(const TileSet& ts, int slot, int gi, int cx, int cy, int cz, long long v) {
    if (slot < 0) return false;
    const DepTile& t = ts.t[slot];
    if (t.gi != gi) return false;
    const unsigned x = (unsigned)(cx - t.o[0]), y = (unsigned)(cy - t.o[1]), z = (unsigned)(cz - t.o[2]);
    if (x >= (unsigned)t.n[0] || y >= (unsigned)t.n[1] || z >= (unsigned)t.n[2]) return false;
    const int k = t.base + (int)x + t.n[0] * ((int)y + t.n[1] * (int)z);
    const unsigned lo = (unsigned)v, hi = (unsigned)((unsigned long long)v >> 32);
    const unsigned old = atomicAdd(ts.lo + k, lo);
    const unsigned add_hi = hi + (old + lo < old ? 1u : 0u);   // the carry out of the low word
    if (add_hi) atomicAdd(ts.hi + k, add_hi);
    return true;
}

// CTA size and minimum resident CTAs per SM of the particle deposit
#ifndef APM_DEP_THREADS
#define APM_DEP_THREADS 128
#endif
#ifndef APM_DEP_MIN_CTAS
#define APM_DEP_MIN_CTAS 6
#endif
constexpr int kDepThreads = APM_DEP_THREADS;
static_assert(kDepThreads % 32 == 0, "the root deposit exchanges charges across whole warps");

template <bool SMALL>
__device__ __forceinline__ unsigned long long mul63(unsigned long long a, unsigned long long b) {
    return SMALL ? wmul63_small(a, b) : wmul63(a, b);
}

// The 27 charges of one particle into every candidate grid [e0, e1) of the
// level: ((|M| wx) wy) wz for the 26 outer cells, every product rounded half up
// on the scale 2^63, the centre cell M minus the others.  SMALL: |M| < 2^32.
template <bool SMALL, bool TILE>
__device__ __forceinline__ void scatter_charges(const LevelDev& L, int64_t* const* __restrict__ gmf,
                                                unsigned* __restrict__ status, long long M,
                                                unsigned long long aM, const unsigned long long w[3][3],
                                                const long long ic[3], int e0, int e1, bool outside,
                                                const TileSet& ts, int slot) {
    unsigned long long mx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) mx[a] = mul63<SMALL>(aM, w[0][a]);
    for (int e = e0; e < e1; ++e) {
        const int gi = L.is_root ? 0 : L.map.dep_list[e];
        const GridDev& g = L.g[gi];
        if (g.mode == 1 && outside) atomicOr(status, kStOutOfBox);
        int64_t* __restrict__ out = gmf[gi];
        // GMF boxes hold fewer than 2^31 cells (checked on the host)
        int cx[3], cy[3], cz[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            cx[k] = edge_rule(ic[0] + k - 1 - g.lo[0], g.G[0], g.mode);
            cy[k] = edge_rule(ic[1] + k - 1 - g.lo[1], g.G[1], g.mode);
            cz[k] = edge_rule(ic[2] + k - 1 - g.lo[2], g.G[2], g.mode);
        }
        const unsigned G0 = g.G[0], G01 = (unsigned)g.G[0] * g.G[1];
        long long others = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            unsigned long long mxy[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) mxy[a] = mul63<SMALL>(mx[a], w[1][b]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const bool ok = cy[b] >= 0 && cz[c] >= 0;
                const unsigned row = G0 * (unsigned)cy[b] + G01 * (unsigned)cz[c];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (a == 1 && b == 1 && c == 1) continue;
                    long long v = (long long)mul63<SMALL>(mxy[a], w[2][c]);
                    v = M < 0 ? -v : v;
                    others += v;
                    if (ok && cx[a] >= 0 && APM_IN_BOUNDS(row + (unsigned)cx[a], g.cells_gmf, status)) {
                        if (!TILE || !tile_add(ts, slot, gi, cx[a], cy[b], cz[c], v))
                            add_charge(out, row + (unsigned)cx[a], v);
                    }
                }
            }
        }
        const unsigned ci = (unsigned)cx[1] + G0 * (unsigned)cy[1] + G01 * (unsigned)cz[1];
        if (cx[1] >= 0 && cy[1] >= 0 && cz[1] >= 0 && APM_IN_BOUNDS(ci, g.cells_gmf, status)) {
            if (!TILE || !tile_add(ts, slot, gi, cx[1], cy[1], cz[1], M - others)) add_charge(out, ci, M - others);
        }
    }
}

// ---- the root level with x neighbours merged across the warp ----
// Particles stored in x order (a lattice such as the Zel'dovich workloads',
// row by row) put lane j's cloud next to lane j-1's along x: at a spacing of
// two cells, lane j-1's column cx+1 is lane j's column cx-1, in the same nine
// (y, z) rows.  Lane j then adds lane j-1's nine column +1 charges to its own
// column (0 or 1) on the same cells, and lane j-1 leaves them out: one 64-bit
// reduction per such cell instead of two.  Integer addition is exact and
// associative, so the field is the same bit for bit.  The partners are tested
// on the cells themselves (all of cy and cz, and lane j-1's cx[2] against
// lane j's cx[0] or cx[1]), so the edge rules (fold, wrap, drop) need no
// special case.  A lane never merges into its column 2, the one it may pass
// on, so no charge is ever forwarded twice.
template <bool SMALL>
__device__ __forceinline__ void scatter_root_merged(const GridDev& g, int64_t* __restrict__ out,
                                                    unsigned* __restrict__ status, long long M,
                                                    unsigned long long aM, const unsigned long long w[3][3],
                                                    const int cx[3], const int cy[3], const int cz[3], bool ok,
                                                    int ma, bool give) {
    constexpr unsigned kFull = 0xffffffffu;
    unsigned long long mx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) mx[a] = mul63<SMALL>(aM, w[0][a]);
    const unsigned G0 = g.G[0], G01 = (unsigned)g.G[0] * g.G[1];
    long long others = 0, centre_in = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        unsigned long long mxy[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) mxy[a] = mul63<SMALL>(mx[a], w[1][b]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            long long v[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == 1 && b == 1 && c == 1) {
                    v[a] = 0;
                    continue;
                }
                long long q = (long long)mul63<SMALL>(mxy[a], w[2][c]);
                q = M < 0 ? -q : q;
                others += q;
                v[a] = q;
            }
            // lane j-1's column 2 of this row (every lane exchanges)
            const long long in = __shfl_up_sync(kFull, v[2], 1);
            if (ma == 0) {
                v[0] += in;
            } else if (ma == 1) {
                if (b == 1 && c == 1) centre_in = in;
                else v[1] += in;
            }
            const bool rok = ok && cy[b] >= 0 && cz[c] >= 0;
            const unsigned row = G0 * (unsigned)cy[b] + G01 * (unsigned)cz[c];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a == 1 && b == 1 && c == 1) continue;
                if (a == 2 && give) continue;
                if (rok && cx[a] >= 0 && APM_IN_BOUNDS(row + (unsigned)cx[a], g.cells_gmf, status))
                    add_charge(out, row + (unsigned)cx[a], v[a]);
            }
        }
    }
    const unsigned ci = (unsigned)cx[1] + G0 * (unsigned)cy[1] + G01 * (unsigned)cz[1];
    if (ok && cx[1] >= 0 && cy[1] >= 0 && cz[1] >= 0 && APM_IN_BOUNDS(ci, g.cells_gmf, status))
        add_charge(out, ci, M - others + centre_in);
}

// The root level's deposit of this lane's particle (fixed-point position X,
// integer mass M; ok false: no particle, the lane only takes part in the
// exchanges).  Every lane of the warp must call it, with none exited.
__device__ __forceinline__ void deposit_root_merged(const LevelDev& L, const long long X[3], long long M,
                                                    bool ok, bool outside, int64_t* const* __restrict__ gmf,
                                                    unsigned* __restrict__ status) {
    constexpr unsigned kFull = 0xffffffffu;
    const GridDev& g = L.g[0];
    const int PB = L.frac_bits;
    long long ic[3];
    unsigned long long w[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        ic[j] = X[j] >> PB;
        tsc_fixed(X[j], PB, w[j]);
    }
    if (ok && g.mode == 1 && outside) atomicOr(status, kStOutOfBox);
    int cx[3], cy[3], cz[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        cx[k] = edge_rule(ic[0] + k - 1 - g.lo[0], g.G[0], g.mode);
        cy[k] = edge_rule(ic[1] + k - 1 - g.lo[1], g.G[1], g.mode);
        cz[k] = edge_rule(ic[2] + k - 1 - g.lo[2], g.G[2], g.mode);
    }
    // lane j-1's cells, exchanged unconditionally (every lane reaches every shuffle)
    const int lane = threadIdx.x & 31;
    const int pok = __shfl_up_sync(kFull, ok ? 1 : 0, 1);
    const int pcx2 = __shfl_up_sync(kFull, cx[2], 1);
    int pcy[3], pcz[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pcy[k] = __shfl_up_sync(kFull, cy[k], 1);
        pcz[k] = __shfl_up_sync(kFull, cz[k], 1);
    }
    bool same = ok && pok != 0 && lane > 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) same = same && pcy[k] == cy[k] && pcz[k] == cz[k];
    // this lane's column that takes lane j-1's column 2 (-1: none)
    const int ma = !same ? -1 : (cx[0] == pcx2 ? 0 : (cx[1] == pcx2 ? 1 : -1));
    // lane j+1 takes this lane's column 2
    const int next_takes = __shfl_down_sync(kFull, ma >= 0 ? 1 : 0, 1);
    const bool give = ok && lane < 31 && next_takes != 0;
    const unsigned long long aM = (unsigned long long)(M < 0 ? -M : M);
    // one product width for the whole warp (the general products round the
    // same way), so that every lane reaches the same shuffles
    if (__all_sync(kFull, !ok || aM < (1ULL << 32)))
        scatter_root_merged<true>(g, gmf[0], status, M, aM, w, cx, cy, cz, ok, ma, give);
    else
        scatter_root_merged<false>(g, gmf[0], status, M, aM, w, cx, cy, cz, ok, ma, give);
}

// Deposit of one particle (fixed-point position X, integer mass M) into the
// grids of one level; false when the particle is not a candidate of the level
// (then it is none of a finer level's either: finer GMF boxes lie inside the
// interiors of their parents).
template <bool TILE>
__device__ __forceinline__ bool deposit_level(const LevelDev& L, const long long X[3], long long M,
                                              bool outside, int64_t* const* __restrict__ gmf,
                                              unsigned* __restrict__ status, const TileSet& ts, int slot) {
    const int PB = L.frac_bits;
    long long ic[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) ic[j] = X[j] >> PB;
    // candidate grids
    int e0 = 0, e1 = 1;
    if (!L.is_root) {
        const TileMap& m = L.map;
        long long t[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            long long rel = ic[j] - m.lo[j];
            if (rel < 0) return false;
            t[j] = rel >> m.shift;
            if (t[j] >= m.nt[j]) return false;
        }
        long long tile = t[0] + (long long)m.nt[0] * (t[1] + (long long)m.nt[1] * t[2]);
        e0 = m.dep_off[tile];
        e1 = m.dep_off[tile + 1];
        if (e0 == e1) return false;
    }
    unsigned long long w[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) tsc_fixed(X[j], PB, w[j]);
    const unsigned long long aM = (unsigned long long)(M < 0 ? -M : M);
    if (aM < (1ULL << 32))   // every product has a 32-bit factor: |M|, then (|M| wx), then (|M| wx) wy
        scatter_charges<true, TILE>(L, gmf, status, M, aM, w, ic, e0, e1, outside, ts, slot);
    else
        scatter_charges<false, TILE>(L, gmf, status, M, aM, w, ic, e0, e1, outside, ts, slot);
    return true;
}

// drifted coordinates, fixed-point position and integer mass of particle p;
// false (and the overflow flag) when |m 2^F| >= 2^62
__device__ __forceinline__ bool particle_fixed(const LevelDev& L, const Particles& P, long long p,
                                               double half_dt, double box, int F, long long X[3],
                                               long long* M, bool* outside, unsigned* __restrict__ status) {
    const double xd[3] = {drift_raw(P.x[p], P.vx[p], half_dt), drift_raw(P.y[p], P.vy[p], half_dt),
                          drift_raw(P.z[p], P.vz[p], half_dt)};
#pragma unroll
    for (int j = 0; j < 3; ++j) X[j] = fixed_position(xd[j], L);   // the same for every level
    bool ok;
    *M = scaled_rint(P.m[p], F, ok);   // rint(m 2^F)
    if (!ok) {
        atomicOr(status, kStOverflow);
        return false;
    }
    // isolated root only: a drifted particle outside [0, box) is flagged (its cloud folds)
    *outside = L.g[0].mode == 1 && L.is_root &&
               !(xd[0] >= 0.0 && xd[0] < box && xd[1] >= 0.0 && xd[1] < box && xd[2] >= 0.0 && xd[2] < box);
    return true;
}

// the first candidate grid of level L for the fixed-point position X (the
// root: grid 0), or -1 when the particle is no candidate of the level
__device__ __forceinline__ int first_candidate(const LevelDev& L, const long long X[3]) {
    if (L.is_root) return 0;
    const TileMap& m = L.map;
    long long t[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const long long rel = (X[j] >> L.frac_bits) - m.lo[j];
        if (rel < 0) return -1;
        t[j] = rel >> m.shift;
        if (t[j] >= m.nt[j]) return -1;
    }
    const long long tile = t[0] + (long long)m.nt[0] * (t[1] + (long long)m.nt[1] * t[2]);
    const int e0 = m.dep_off[tile];
    return e0 == m.dep_off[tile + 1] ? -1 : m.dep_list[e0];
}

// the box of tile slot `slot` on absolute level `lev` for bins of 2^shift root
// cells: the bin and the next along x, one cell of halo (extents n); false
// when the slots up to this one exceed kTileCells
__device__ __forceinline__ bool tile_extent(int lev, int shift, int n[3], int& cells) {
    if (shift + lev > 10) return false;
    const int b = 1 << (shift + lev);
    n[0] = 2 * b + 2;
    n[1] = n[2] = b + 2;
    cells = n[0] * n[1] * n[2];
    return true;
}

// tile set-up of a CTA over levels lv[0..nl) (the levels in slot order): the
// layout (every thread), then the anchor of each slot (the CTA's first
// particle that is a candidate of its level) and, by that thread, the grid
// and origin; returns the number of slots and the words used
template <class LV>
__device__ __forceinline__ int tile_setup(const TileSet& ts, int* anchor, const LV& lv, int nl, int shift, bool ok,
                                          const long long X[3], int& used) {
    int nslots = 0;
    used = 0;
    for (int l = 0; l < nl && l < kMaxTileLevels; ++l) {
        int n[3], cells;
        if (!tile_extent(lv(l).level, shift, n, cells) || used + cells > kTileCells) break;
        if (threadIdx.x == 0) {
            DepTile& t = ts.t[l];
            t.gi = -1;
            t.n[0] = n[0];
            t.n[1] = n[1];
            t.n[2] = n[2];
            t.base = used;
            anchor[l] = INT_MAX;
        }
        used += cells;
        ++nslots;
    }
    for (int k = threadIdx.x; k < used; k += blockDim.x) {
        ts.lo[k] = 0u;
        ts.hi[k] = 0u;
    }
    __syncthreads();
    if (ok)
        for (int l = 0; l < nslots; ++l) {
            if (first_candidate(lv(l), X) < 0) break;
            atomicMin(anchor + l, (int)threadIdx.x);
        }
    __syncthreads();
    if (ok)
        for (int l = 0; l < nslots; ++l)
            if (anchor[l] == (int)threadIdx.x) {
                const LevelDev& L = lv(l);
                const int gi = first_candidate(L, X);
                const GridDev& g = L.g[gi];
                DepTile& t = ts.t[l];
                t.gi = gi;
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    t.o[j] = (int)(((X[j] >> (kPosBits + shift)) << (shift + L.level)) - g.lo[j]) - 1;
            }
    __syncthreads();
    return nslots;
}

// one reduction per nonzero tile cell (after a barrier that follows every charge)
template <class LV, class GM>
__device__ __forceinline__ void tile_flush(const TileSet& ts, int nslots, int used, const LV& lv, const GM& gm) {
    for (int k = threadIdx.x; k < used; k += blockDim.x) {
        int l = 0;
        while (l + 1 < nslots && k >= ts.t[l + 1].base) ++l;
        const DepTile& t = ts.t[l];
        const unsigned long long v = ((unsigned long long)ts.hi[k] << 32) | ts.lo[k];
        if (t.gi < 0 || v == 0ULL) continue;
        const int r = k - t.base;
        const int x = r % t.n[0], y = (r / t.n[0]) % t.n[1], z = r / (t.n[0] * t.n[1]);
        const GridDev& g = lv(l).g[t.gi];
        const unsigned idx = (unsigned)(t.o[0] + x) + (unsigned)g.G[0] * ((unsigned)(t.o[1] + y) +
                                                                           (unsigned)g.G[1] * (unsigned)(t.o[2] + z));
        add_charge(gm(l)[t.gi], idx, (long long)v);
    }
}

// the deposit of slot i's particle into one level (the candidate test first
// on refined levels: most particles leave there)
template <bool TILE>
__device__ __forceinline__ void deposit_one(const LevelDev& L, const Particles& P, long long i, double half_dt,
                                            double box, int F, int64_t* const* __restrict__ gmf,
                                            unsigned* __restrict__ status, const TileSet& ts, int slot) {
    const long long p = P.at(i);
    long long X[3], M;
    bool outside;
    if (!L.is_root) {
        const double xd[3] = {drift_raw(P.x[p], P.vx[p], half_dt), drift_raw(P.y[p], P.vy[p], half_dt),
                              drift_raw(P.z[p], P.vz[p], half_dt)};
#pragma unroll
        for (int j = 0; j < 3; ++j) X[j] = fixed_position(xd[j], L);
        if (first_candidate(L, X) < 0) return;
        bool ok;
        M = scaled_rint(P.m[p], F, ok);
        if (!ok) {
            atomicOr(status, kStOverflow);
            return;
        }
        deposit_level<TILE>(L, X, M, false, gmf, status, ts, slot);
        return;
    }
    if (!particle_fixed(L, P, p, half_dt, box, F, X, &M, &outside, status)) return;
    deposit_level<TILE>(L, X, M, outside, gmf, status, ts, slot);
}

// TILE: the particles are in bin order, and each CTA gathers the charges of
// its bin in shared memory (see tile_add)
template <bool TILE>
__global__ void __launch_bounds__(kDepThreads, APM_DEP_MIN_CTAS) k_deposit(LevelDev L, Particles P, double half_dt,
                                                 double box, int F,
                                                 int64_t* const* __restrict__ gmf,
                                                 unsigned* __restrict__ status) {
    __shared__ unsigned t_lo[TILE ? kTileCells : 1], t_hi[TILE ? kTileCells : 1];
    __shared__ DepTile tiles[TILE ? kMaxTileLevels : 1];
    __shared__ int anchor[TILE ? kMaxTileLevels : 1];
    const TileSet ts{tiles, t_lo, t_hi};
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if constexpr (!TILE) {
        if (i < P.n) deposit_one<false>(L, P, i, half_dt, box, F, gmf, status, ts, -1);
    } else {
        // the anchor's position: drifted and fixed like the deposit's (the
        // candidate and mass checks follow in deposit_one)
        long long X[3] = {0, 0, 0};
        const bool live = i < P.n;
        if (live) {
            const long long p = P.at(i);
            const double xd[3] = {drift_raw(P.x[p], P.vx[p], half_dt), drift_raw(P.y[p], P.vy[p], half_dt),
                                  drift_raw(P.z[p], P.vz[p], half_dt)};
#pragma unroll
            for (int j = 0; j < 3; ++j) X[j] = fixed_position(xd[j], L);
        }
        auto lv = [&](int) -> const LevelDev& { return L; };
        int used;
        const int nslots = tile_setup(ts, anchor, lv, 1, P.order_shift, live, X, used);
        if (live) deposit_one<true>(L, P, i, half_dt, box, F, gmf, status, ts, nslots > 0 ? 0 : -1);
        __syncthreads();
        tile_flush(ts, nslots, used, lv, [&](int) { return gmf; });
    }
}

// Every level in one pass over the particles: the position and mass are
// converted once, then deposited level by level from the root down while the
// particle is a candidate.  levels: the LevelDev of each level; gmfs[l]: the
// GMF pointer table of level l.
template <bool TILE>
__global__ void __launch_bounds__(kDepThreads, APM_DEP_MIN_CTAS) k_deposit_levels(
    const LevelDev* __restrict__ levels, int nl, Particles P, double half_dt, double box, int F,
    int64_t* const* const* __restrict__ gmfs, unsigned* __restrict__ status) {
    __shared__ unsigned t_lo[TILE ? kTileCells : 1], t_hi[TILE ? kTileCells : 1];
    __shared__ DepTile tiles[TILE ? kMaxTileLevels : 1];
    __shared__ int anchor[TILE ? kMaxTileLevels : 1];
    const TileSet ts{tiles, t_lo, t_hi};
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long X[3] = {0, 0, 0}, M = 0;
    bool outside = false, ok = false;
    if (i < P.n) ok = particle_fixed(levels[0], P, P.at(i), half_dt, box, F, X, &M, &outside, status);
    int nslots = 0, used = 0;
    auto lv = [&](int l) -> const LevelDev& { return levels[l]; };
    if constexpr (TILE) nslots = tile_setup(ts, anchor, lv, nl, P.order_shift, ok, X, used);
    int l0 = 0;
    if constexpr (!TILE) {
        // the root with the warp's x neighbours merged: every lane, with or
        // without a particle (blocks are whole warps)
        if (levels[0].is_root) {
            deposit_root_merged(levels[0], X, M, ok, outside, gmfs[0], status);
            l0 = 1;
        }
    }
    if (ok)
        for (int l = l0; l < nl; ++l)
            if (!deposit_level<TILE>(levels[l], X, M, l == 0 && outside, gmfs[l], status, ts, l < nslots ? l : -1))
                break;
    if constexpr (TILE) {
        __syncthreads();
        tile_flush(ts, nslots, used, lv, [&](int l) { return gmfs[l]; });
    }
}

}  // namespace

cudaError_t launch_gas_init(const LevelDev& L, const GridDev* parent_grids,
                            const double* const* gas, const double* const* pgas,
                            int64_t* const* gmf, const Chunk* chunks, int n_chunks,
                            int F, cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    k_gas_init<<<n_chunks, 256, 0, s>>>(L, parent_grids, gas, pgas, gmf, chunks, F);
    return cudaGetLastError();
}

cudaError_t launch_deposit(const LevelDev& L, const Particles& P, double half_dt, double box,
                           int F, int64_t* const* gmf, unsigned* status, cudaStream_t s) {
    if (P.n <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((P.n + kDepThreads - 1) / kDepThreads);
    if (P.perm)
        k_deposit<true><<<blocks, kDepThreads, 0, s>>>(L, P, half_dt, box, F, gmf, status);
    else
        k_deposit<false><<<blocks, kDepThreads, 0, s>>>(L, P, half_dt, box, F, gmf, status);
    return cudaGetLastError();
}

cudaError_t launch_deposit_levels(const LevelDev* levels, int nl, const Particles& P, double half_dt,
                                  double box, int F, int64_t* const* const* gmfs, unsigned* status,
                                  cudaStream_t s) {
    if (P.n <= 0 || nl <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((P.n + kDepThreads - 1) / kDepThreads);
    if (P.perm)
        k_deposit_levels<true><<<blocks, kDepThreads, 0, s>>>(levels, nl, P, half_dt, box, F, gmfs, status);
    else
        k_deposit_levels<false><<<blocks, kDepThreads, 0, s>>>(levels, nl, P, half_dt, box, F, gmfs, status);
    return cudaGetLastError();
}

}  // namespace apm

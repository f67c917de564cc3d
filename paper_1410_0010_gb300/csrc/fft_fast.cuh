// fft_fast.cuh -- FP32 FFT passes with the transform length and its radices
// fixed at compile time (the lengths of fast_radices()), for the same five
// passes, work lists and data layout as fft_core.cuh's runtime-planned
// kernels, which remain the path for every other length and for FP64.
//
// A length L = R1 R2 (R3) is transformed in place in ONE shared-memory
// buffer, element-major (line fastest):
//   forward: decimation in frequency.  Element n = n1 R2 R3 + n2 R3 + n3 sits
//     at position n.  Stage s takes a DFT of radix R_s over digit s of the
//     position and multiplies its output k by exp(-2 pi i lo k / (R_s S_s))
//     (S_s = product of the radices after s, lo = the digits after s), in
//     place; after the last stage the spectrum X[k1 + R1 k2 + R1 R2 k3]
//     sits at position (k1, k2, k3) (digit-reversed order).
//   inverse: decimation in time, the forward's exact reverse: stages from the
//     last digit to the first, each multiplying by the conjugate twiddles
//     before its inverse DFT; it takes the digit-reversed spectrum and leaves
//     the signal in natural order.
// A butterfly reads and writes the same R positions, so no second buffer is
// needed; the first stage reads its inputs straight from HBM and the last
// stage writes straight to HBM, with the natural element index computed from
// the digits.  Every index, trip count and twiddle stride is a compile-time
// constant except the butterfly number of the thread.
#pragma once
#include "fft_core.cuh"

namespace apm {
namespace {

// DFT of radix R in registers: the building blocks of fft_core.cuh (direct
// radices 2, 3, 4, 5, 7, 8 and composites R1 x R2)
template <int DIR, int R> struct FastDft;
#define APM_FAST_DFT_DIRECT(R) \
    template <int DIR> struct FastDft<DIR, R> { \
        __device__ __forceinline__ static void run(float2* v) { Dft<float, DIR, R>::run(v); } \
    };
#define APM_FAST_DFT_COMPOSITE(R, A, B) \
    template <int DIR> struct FastDft<DIR, R> { \
        __device__ __forceinline__ static void run(float2* v) { DftC<float, DIR, A, B>::run(v); } \
    };
APM_FAST_DFT_DIRECT(2)
APM_FAST_DFT_DIRECT(3)
APM_FAST_DFT_DIRECT(4)
APM_FAST_DFT_DIRECT(5)
APM_FAST_DFT_DIRECT(7)
APM_FAST_DFT_DIRECT(8)
APM_FAST_DFT_COMPOSITE(6, 3, 2)
APM_FAST_DFT_COMPOSITE(9, 3, 3)
APM_FAST_DFT_COMPOSITE(10, 5, 2)
APM_FAST_DFT_COMPOSITE(12, 3, 4)
APM_FAST_DFT_COMPOSITE(14, 7, 2)
APM_FAST_DFT_COMPOSITE(15, 5, 3)
APM_FAST_DFT_COMPOSITE(16, 4, 4)
#undef APM_FAST_DFT_DIRECT
#undef APM_FAST_DFT_COMPOSITE

// The compile-time plan: radices R1, R2, R3 (R3 = 1 for two stages).
template <int A, int B, int Cc> struct FastPlan {
    static constexpr int R1 = A, R2 = B, R3 = Cc;
    static constexpr int L = A * B * Cc;
    static constexpr int NST = Cc == 1 ? 2 : 3;
    // radix and inner stride of stage s (0-based)
    static constexpr int radix(int s) { return s == 0 ? A : (s == 1 ? B : Cc); }
    static constexpr int inner(int s) { return s == 0 ? B * Cc : (s == 1 ? Cc : 1); }
    // natural (frequency) index of the digit-reversed position with digits
    // (d1, d2, d3): d1 + R1 d2 + R1 R2 d3
    __device__ __forceinline__ static int natural(int pos) {
        const int d1 = pos / (B * Cc), rest = pos - d1 * (B * Cc);
        const int d2 = rest / Cc, d3 = rest - d2 * Cc;
        return d1 + A * d2 + A * B * d3;
    }
    // the natural-index weight of the last digit: in the last stage (inner
    // stride 1) a butterfly's element k sits at position base + k, and its
    // natural index is natural(base) + k last_weight()
    static constexpr int last_weight() { return L / radix(NST - 1); }
    // the position of natural index k (the inverse of natural())
    __device__ __forceinline__ static int position(int k) {
        const int d1 = k % A, q = k / A;
        const int d2 = q % B, d3 = q / B;
        return d1 * (B * Cc) + d2 * Cc + d3;
    }
};

// One DIF stage s over TX lines with NT threads (line l of position p at
// buf[p PITCH + l]): butterfly b = (hi, lo) of the
// stage's L / R butterflies per line reads positions hi R S + k S + lo, takes
// the DFT (DIR -1 forward; +1 the unnormalised inverse, with conjugate
// twiddles) and multiplies output k by tw[lo k L / (R S)] (or its conjugate).
//  IN_G: the inputs come from global memory (natural index = position)
//  OUT_G: the outputs go to global memory (natural index from the digits;
//         only for the last stage, whose digits are complete)
template <class P, int S_, int TX, int NT, bool IN_G, bool OUT_G, class GIN, class GOUT, int PITCH = TX,
          int DIR = -1>
__device__ __forceinline__ void fast_dif_stage(float2* buf, const float2* __restrict__ tw, const GIN& gin,
                                               const GOUT& gout) {
    constexpr int R = P::radix(S_), S = P::inner(S_), L = P::L;
    constexpr int NB = L / R, ITEMS = NB * TX, TRIPS = (ITEMS + NT - 1) / NT;
    constexpr int TWS = L / (R * S);
#pragma unroll
    for (int it = 0; it < TRIPS; ++it) {
        const int i = threadIdx.x + it * NT;
        if (ITEMS % NT != 0 && i >= ITEMS) break;
        const int line = i % TX, b = i / TX;
        const int hi = b / S, lo = b - hi * S;
        const int base = hi * R * S + lo;
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (IN_G) v[k] = gin.ld(base + k * S);
            else v[k] = buf[(base + k * S) * PITCH + line];
        }
        FastDft<DIR, R>::run(v);
        if constexpr (S > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = mul<float>(v[k], twid<float, DIR>(tw, lo * k * TWS));
        }
        static_assert(!OUT_G || S == 1, "global output only from the last stage");
        const int nat0 = OUT_G ? P::natural(base) : 0;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (OUT_G) gout.st(nat0 + k * P::last_weight(), v[k]);
            else buf[(base + k * S) * PITCH + line] = v[k];
        }
    }
}

// One DIT (inverse) stage s: butterfly (hi, lo) multiplies input k by
// conj(tw[lo k L / (R S)]), takes the inverse DFT and writes output r to
// position hi R S + r S + lo.
//  IN_G: the inputs come from global memory (natural index from the digits;
//        only for the first inverse stage, the last digit)
//  OUT_G: the outputs go to global memory (the first digit's stage: the
//         positions are then natural indices)
template <class P, int S_, int TX, int NT, bool IN_G, bool OUT_G, class GIN, class GOUT, int PITCH = TX>
__device__ __forceinline__ void fast_dit_stage(float2* buf, const float2* __restrict__ tw, const GIN& gin,
                                               const GOUT& gout) {
    constexpr int R = P::radix(S_), S = P::inner(S_), L = P::L;
    constexpr int NB = L / R, ITEMS = NB * TX, TRIPS = (ITEMS + NT - 1) / NT;
    constexpr int TWS = L / (R * S);
#pragma unroll
    for (int it = 0; it < TRIPS; ++it) {
        const int i = threadIdx.x + it * NT;
        if (ITEMS % NT != 0 && i >= ITEMS) break;
        const int line = i % TX, b = i / TX;
        const int hi = b / S, lo = b - hi * S;
        const int base = hi * R * S + lo;
        float2 v[R];
        static_assert(!IN_G || S == 1, "global input only to the first inverse stage");
        const int nat0 = IN_G ? P::natural(base) : 0;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (IN_G) v[k] = gin.ld(nat0 + k * P::last_weight());
            else v[k] = buf[(base + k * S) * PITCH + line];
        }
        if constexpr (S > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = mul<float>(v[k], twid<float, 1>(tw, lo * k * TWS));
        }
        FastDft<1, R>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (OUT_G) gout.st(base + k * S, v[k]);
            else buf[(base + k * S) * PITCH + line] = v[k];
        }
    }
}

// The z pass's middle: the forward's last stage (S = 1), the table multiply at
// the natural index, and the inverse's first stage on the same registers.
template <class P, int TX, int NT, class TAB>
__device__ __forceinline__ void fast_mid_stage(float2* buf, const TAB& tabf) {
    constexpr int SL = P::NST - 1;
    constexpr int R = P::radix(SL), L = P::L;
    constexpr int NB = L / R, ITEMS = NB * TX, TRIPS = (ITEMS + NT - 1) / NT;
#pragma unroll
    for (int it = 0; it < TRIPS; ++it) {
        const int i = threadIdx.x + it * NT;
        if (ITEMS % NT != 0 && i >= ITEMS) break;
        const int line = i % TX, hi = i / TX;
        const int base = hi * R;
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = buf[(base + k) * TX + line];
        FastDft<-1, R>::run(v);
        // natural index of output k: the digits of hi, then k as the last digit
        const int k0 = P::natural(base);
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = tabf.apply(k0 + k * (L / R), v[k]);
        FastDft<1, R>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) buf[(base + k) * TX + line] = v[k];
    }
}

// Global element n of this thread's line: p[n stride] for n < n_in (zero
// beyond: the padding); nothing for a dead line (kx >= Hx).  Offsets stay
// 32-bit (lines of at most 1024 elements, strides below 1024 x 513).
struct FastIn {
    const float2* __restrict__ p;
    int stride, n;
    bool live;
    __device__ __forceinline__ float2 ld(int i) const {
        return (live && i < n) ? p[i * stride] : make_float2(0.f, 0.f);
    }
};
// Output element i at window index w = (i - s0) mod L, written when w < n, and
// again at w + L when that is inside the window too (a periodic root's window
// N + 4 exceeds M = N).
template <int L> struct FastOut {
    float2* __restrict__ p;
    int stride, n, s0;
    bool live;
    __device__ __forceinline__ void st(int i, float2 v) const {
        if (!live) return;
        int w = i - s0;
        if (w < 0) w += L;
        if (w < n) p[w * stride] = v;
        if (w + L < n) p[(w + L) * stride] = v;
    }
};

// Output element i of a pass with no window (the y forward: all L outputs)
struct FastOutAll {
    float2* __restrict__ p;
    int stride;
    bool live;
    __device__ __forceinline__ void st(int i, float2 v) const {
        if (live) p[i * stride] = v;
    }
};

// Column pass (AX 1: y, 2: z) with compile-time plan P, TX kx columns per CTA
// (the level's lines for this pass) and NT threads; the same work list and
// layout as k_col (MODE 0 yf, 1 z with the table, 2 yi, 3 z with the table
// times -i D_comp of spectral-gradient component comp).
template <class P, int AX, int MODE, int TX, int NT>
__global__ void __launch_bounds__(NT) k_col_fast(const GridDev* __restrict__ grids, const Chunk* __restrict__ chunks,
                                                 const float2* __restrict__ tw_arena, const float* __restrict__ tab,
                                                 float2* __restrict__ wsA, float2* __restrict__ wsB, int comp) {
    constexpr int L = P::L;
    extern __shared__ __align__(16) unsigned char smem_fast[];
    float2* buf = reinterpret_cast<float2*>(smem_fast);
    float2* tw = buf + L * TX;
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    const int Hx = g.Hx;
    const int other = ch.tile & ((1 << kColOtherBits) - 1);
    const int kx0 = (ch.tile >> kColOtherBits) * TX;
    const FftPlan1D& pl = AX == 1 ? g.fy : g.fz;
    for (int t = threadIdx.x; t < L; t += NT) tw[t] = tw_arena[pl.tw_off + t];
    const int M1 = g.M[1];

    // global accessors of this thread's line: with NT a multiple of TX the line
    // (threadIdx.x % TX) is the same in every trip of every stage
    static_assert(NT % TX == 0, "NT must be a multiple of TX");
    const int line = threadIdx.x % TX;
    const bool live = kx0 + line < Hx;
    FastIn gin;
    FastOut<L> gout;
    gin.live = gout.live = live;
    if (AX == 1 && MODE == 0) {
        gin.p = wsA + (g.wsA + (long long)other * g.G[1] * Hx + kx0 + line);
        gin.stride = Hx; gin.n = g.G[1];
        gout.p = wsB + (g.wsB + (long long)other * M1 * Hx + kx0 + line);
        gout.stride = Hx; gout.n = M1; gout.s0 = 0;
    } else if (AX == 2) {
        gin.p = wsB + (g.wsB + (long long)other * Hx + kx0 + line);
        gin.stride = M1 * Hx; gin.n = g.G[2];
        gout.p = wsA + (g.wsA + (long long)other * Hx + kx0 + line);
        gout.stride = M1 * Hx; gout.n = g.W[2]; gout.s0 = g.s0[2];
    } else {
        gin.p = wsA + (g.wsA + (long long)other * M1 * Hx + kx0 + line);
        gin.stride = Hx; gin.n = M1;
        gout.p = wsB + (g.wsB + (long long)other * g.W[1] * Hx + kx0 + line);
        gout.stride = Hx; gout.n = g.W[1]; gout.s0 = g.s0[1];
    }
    __syncthreads();   // twiddles

    if constexpr (MODE == 0) {
        // the y forward writes all M1 outputs: no window test
        const FastOutAll gall{gout.p, gout.stride, live};
        if constexpr (P::NST == 2) {
            fast_dif_stage<P, 0, TX, NT, true, false>(buf, tw, gin, gall);
            __syncthreads();
            fast_dif_stage<P, 1, TX, NT, false, true>(buf, tw, gin, gall);
        } else {
            fast_dif_stage<P, 0, TX, NT, true, false>(buf, tw, gin, gall);
            __syncthreads();
            fast_dif_stage<P, 1, TX, NT, false, false>(buf, tw, gin, gall);
            __syncthreads();
            fast_dif_stage<P, 2, TX, NT, false, true>(buf, tw, gin, gall);
        }
    } else if constexpr (MODE == 2) {
        if constexpr (P::NST == 2) {
            fast_dit_stage<P, 1, TX, NT, true, false>(buf, tw, gin, gout);
            __syncthreads();
            fast_dit_stage<P, 0, TX, NT, false, true>(buf, tw, gin, gout);
        } else {
            fast_dit_stage<P, 2, TX, NT, true, false>(buf, tw, gin, gout);
            __syncthreads();
            fast_dit_stage<P, 1, TX, NT, false, false>(buf, tw, gin, gout);
            __syncthreads();
            fast_dit_stage<P, 0, TX, NT, false, true>(buf, tw, gin, gout);
        }
    } else {
        // phi-hat = T(kappa) rho-hat between the forward and the inverse
        // (MODE 1); MODE 3, a spectral-gradient component comp (1-3):
        // -i D_comp T(kappa) rho-hat
        const int ky = other;
        const int fy = ky <= M1 / 2 ? ky : M1 - ky;
        TabCol<float> tabc;   // a dead line reads column 0 (its results are never stored)
        tabc.p = tab + (g.tab_off + (long long)fy * Hx + (live ? kx0 + line : 0));
        tabc.zst = g.Hy2 * Hx;
        tabc.L = L;
        using Tab = typename std::conditional<MODE == 3, TabGrad<float>, TabCol<float>>::type;
        Tab tabf;
        if constexpr (MODE == 3) {
            const int kx = kx0 + line;
            tabf.tab = tabc;
            tabf.comp = comp;
            tabf.dz = (float)g.dk[2];
            const int M0 = g.M[0];
            const int kyc = ky <= M1 / 2 ? ky : ky - M1;
            tabf.dline = comp == 1 ? (2 * kx == M0 ? 0.f : (float)(g.dk[0] * kx))
                                   : (comp == 2 ? (2 * ky == M1 ? 0.f : (float)(g.dk[1] * kyc)) : 0.f);
        } else {
            tabf = tabc;
        }
        fast_dif_stage<P, 0, TX, NT, true, false>(buf, tw, gin, gout);
        __syncthreads();
        if constexpr (P::NST == 3) {
            fast_dif_stage<P, 1, TX, NT, false, false>(buf, tw, gin, gout);
            __syncthreads();
        }
        fast_mid_stage<P, TX, NT>(buf, tabf);
        __syncthreads();
        if constexpr (P::NST == 3) {
            fast_dit_stage<P, 1, TX, NT, false, false>(buf, tw, gin, gout);
            __syncthreads();
        }
        fast_dit_stage<P, 0, TX, NT, false, true>(buf, tw, gin, gout);
    }
}

// ---- x-forward pass -------------------------------------------------------------
// A CTA holds NP complex lines, each packing two real rows (2p, 2p+1) of the
// grid (two-for-one real transforms); buffer element (position, line) at
// pos (NP + 1) + line (the padding keeps the row-wise passes conflict-free).
struct NoIO {
    __device__ float2 ld(int) const { return make_float2(0.f, 0.f); }
    __device__ void st(int, float2) const {}
};

// xf: GMF rows -> half spectra along x, A[z][y][kx] (the layout of k_xf).
// Load pass: the CTA's rows are one contiguous int64 range, read with
// consecutive threads on consecutive pairs of cells of a row pair and
// converted (hardware int64 -> float rounding, exact power-of-two scale);
// positions past G0 and missing rows are zero.  Then the forward stages in place, and the separation of the
// two real rows, A_k = (Z_k + conj Z_{L-k}) / 2, B_k = (Z_k - conj Z_{L-k}) / 2i,
// written with consecutive threads on consecutive kx.
template <class P, int NP, int NT>
__global__ void __launch_bounds__(NT) k_xf_fast(const GridDev* __restrict__ grids, const Chunk* __restrict__ chunks,
                                                const int64_t* const* __restrict__ gmf,
                                                const float2* __restrict__ tw_arena, float2* __restrict__ wsA,
                                                int F) {
    constexpr int L = P::L, PITCH = NP + 1, H = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_fast[];
    float2* buf = reinterpret_cast<float2*>(smem_fast);
    float2* tw = buf + L * PITCH;
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    const int G0 = g.G[0];
    const long long r_first = 2LL * ch.tile * NP;
    const int nr = (int)min(2LL * NP, (long long)g.G[1] * g.G[2] - r_first);
    const int64_t* __restrict__ in = gmf[ch.grid] + r_first * G0;
    for (int t = threadIdx.x; t < L; t += NT) tw[t] = tw_arena[g.fx.tw_off + t];
    const float scale = pow2_neg<float>(F);
    // element (x, line p) = (row 2p, row 2p + 1) at x; one thread per pair of
    // positions of a line, with 16-byte loads of both rows when G0 is even
    {
        constexpr int HALF = (L + 1) / 2;
        const bool vec = !(G0 & 1) && !(reinterpret_cast<size_t>(in) & 15);
#pragma unroll 4
        for (int i = threadIdx.x; i < NP * HALF; i += NT) {
            const int p = i / HALF, x = 2 * (i - p * HALF);
            const int q = 2 * p;
            const int64_t* r0 = in + (long long)q * G0 + x;
            long long a0 = 0, a1 = 0, b0 = 0, b1 = 0;
            if (vec && x < G0) {   // G0 even: x + 1 < G0 too
                if (q < nr) {
                    const longlong2 u = *reinterpret_cast<const longlong2*>(r0);
                    a0 = u.x;
                    a1 = u.y;
                }
                if (q + 1 < nr) {
                    const longlong2 w = *reinterpret_cast<const longlong2*>(r0 + G0);
                    b0 = w.x;
                    b1 = w.y;
                }
            } else {
                const bool x0 = x < G0, x1 = x + 1 < G0;
                if (q < nr) {
                    if (x0) a0 = r0[0];
                    if (x1) a1 = r0[1];
                }
                if (q + 1 < nr) {
                    if (x0) b0 = r0[G0];
                    if (x1) b1 = r0[G0 + 1];
                }
            }
            buf[x * PITCH + p] = make_float2(fixed_to_real<float>(a0, scale), fixed_to_real<float>(b0, scale));
            if (L % 2 == 0 || x + 1 < L)
                buf[(x + 1) * PITCH + p] =
                    make_float2(fixed_to_real<float>(a1, scale), fixed_to_real<float>(b1, scale));
        }
    }
    __syncthreads();
    const NoIO none;
    fast_dif_stage<P, 0, NP, NT, false, false, NoIO, NoIO, PITCH>(buf, tw, none, none);
    __syncthreads();
    fast_dif_stage<P, 1, NP, NT, false, false, NoIO, NoIO, PITCH>(buf, tw, none, none);
    __syncthreads();
    if constexpr (P::NST == 3) {
        fast_dif_stage<P, 2, NP, NT, false, false, NoIO, NoIO, PITCH>(buf, tw, none, none);
        __syncthreads();
    }
    float2* __restrict__ out = wsA + (g.wsA + r_first * H);
    for (int f = threadIdx.x; f < NP * H; f += NT) {
        const int p = f / H, k = f - p * H;
        const int q0 = 2 * p;
        if (q0 >= nr) continue;
        const float2 z = buf[P::position(k) * PITCH + p];
        const float2 zm = buf[P::position(k == 0 ? 0 : L - k) * PITCH + p];
        out[q0 * H + k] = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
        if (q0 + 1 < nr) out[(q0 + 1) * H + k] = make_float2(0.5f * (z.y + zm.y), 0.5f * (zm.x - z.x));
    }
}

// ---- x-inverse pass ---------------------------------------------------------------
// One DIF stage s with the butterflies of a line on consecutive threads (item
// i: butterfly i % NB, line i / NB), so the HBM accesses of the first and last
// stages run along rows; buffer element (position e, line) at
// rows_index(e) + line = e PITCH + e / R_last + line.  The last stage's lanes
// step through positions R_last apart: with PITCH odd, one extra element
// every R_last positions makes that stride odd too (R_last PITCH + 1), so a
// half-warp's 64-bit accesses fall in distinct bank pairs (with R_last = 16
// and no padding, all sixteen hit one pair).
// The global accessors take the line: gin.ld(line, n), gout.st(line, n, v).
template <class P, int PITCH>
__device__ __forceinline__ int rows_index(int e) {
    return e * PITCH + e / P::radix(P::NST - 1);
}
template <class P, int S_, int NL, int NT, bool IN_G, bool OUT_G, int DIR, int PITCH, class GIN, class GOUT>
__device__ __forceinline__ void fast_dif_stage_rows(float2* buf, const float2* __restrict__ tw, const GIN& gin,
                                                    const GOUT& gout) {
    constexpr int R = P::radix(S_), S = P::inner(S_), L = P::L;
    constexpr int NB = L / R, ITEMS = NB * NL, TRIPS = (ITEMS + NT - 1) / NT;
    constexpr int TWS = L / (R * S);
#pragma unroll 1
    for (int it = 0; it < TRIPS; ++it) {
        const int i = threadIdx.x + it * NT;
        if (ITEMS % NT != 0 && i >= ITEMS) break;
        const int line = i / NB, b = i - line * NB;
        const int hi = b / S, lo = b - hi * S;
        const int base = hi * R * S + lo;
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (IN_G) v[k] = gin.ld(line, base + k * S);
            else v[k] = buf[rows_index<P, PITCH>(base + k * S) + line];
        }
        FastDft<DIR, R>::run(v);
        if constexpr (S > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = mul<float>(v[k], twid<float, DIR>(tw, lo * k * TWS));
        }
        static_assert(!OUT_G || S == 1, "global output only from the last stage");
        const int nat0 = OUT_G ? P::natural(base) : 0;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (OUT_G) gout.st(line, nat0 + k * P::last_weight(), v[k]);
            else buf[rows_index<P, PITCH>(base + k * S) + line] = v[k];
        }
    }
}

// xi: half spectra -> real rows of the window, C2R two rows per complex line,
// as an in-place decimation-in-frequency inverse (DIR +1).  The first stage
// reads line p's inputs in natural order straight from HBM: Z_k = A_k + i B_k
// (A, B the half spectra of rows 2p, 2p+1), extended by Hermitian symmetry
// (A_{L-k} = conj A_k) past H.  The last stage writes straight to the window:
// real part to row 2p, imaginary part to row 2p+1, at window cell
// w = (x - s0) mod L (and w + L when inside the window), times 1/(M0 M1 M2);
// with a two-stage plan its neighbouring butterflies write neighbouring x.
template <int L> struct XiRowsIn {
    const float2* __restrict__ p;    // row 0 of this CTA
    int nr;                          // rows of this CTA
    __device__ __forceinline__ float2 ld(int line, int k) const {
        constexpr int H = L / 2 + 1;
        const int kk = k < H ? k : L - k;
        const float2* row = p + (2 * line) * H;
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (2 * line < nr) a = row[kk];
        if (2 * line + 1 < nr) b = row[H + kk];
        if (k >= H) {
            a.y = -a.y;
            b.y = -b.y;
        }
        return make_float2(a.x - b.y, a.y + b.x);
    }
};
template <int L> struct XiRowsOut {
    float* __restrict__ p;           // row 0 of this CTA in the window
    int W0, s0, nr;
    float norm;
    __device__ __forceinline__ void st(int line, int x, float2 v) const {
        float* row = p + (2 * line) * W0;
        int w = x - s0;
        if (w < 0) w += L;
        for (; w < W0; w += L) {
            if (2 * line < nr) row[w] = v.x * norm;
            if (2 * line + 1 < nr) row[W0 + w] = v.y * norm;
        }
    }
};

template <class P, int NP, int NT>
__global__ void __launch_bounds__(NT) k_xi_fast(const GridDev* __restrict__ grids, const Chunk* __restrict__ chunks,
                                                const float2* __restrict__ tw_arena,
                                                const float2* __restrict__ wsB, void* const* __restrict__ phis,
                                                int comp) {
    constexpr int L = P::L, H = L / 2 + 1, PITCH = NP + 1;
    extern __shared__ __align__(16) unsigned char smem_fast[];
    float2* buf = reinterpret_cast<float2*>(smem_fast);
    float2* tw = buf + rows_index<P, PITCH>(L);   // past the padded line buffer (<= L PITCH + L / 2)
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    const int W0 = g.W[0];
    const long long r_first = 2LL * ch.tile * NP;
    const int nr = (int)min(2LL * NP, (long long)g.W[1] * g.W[2] - r_first);
    for (int t = threadIdx.x; t < L; t += NT) tw[t] = tw_arena[g.fx.tw_off + t];
    XiRowsIn<L> gin;
    gin.p = wsB + (g.wsB + r_first * H);
    gin.nr = nr;
    XiRowsOut<L> gout;
    // component comp of a spectral-gradient solve: the comp-th window of W cells
    gout.p = reinterpret_cast<float*>(phis[ch.grid]) + (long long)comp * g.W[0] * g.W[1] * g.W[2] + r_first * W0;
    gout.W0 = W0;
    gout.s0 = g.s0[0];
    gout.nr = nr;
    gout.norm = (float)g.inv_m3;
    __syncthreads();   // twiddles
    using GI = XiRowsIn<L>;
    using GO = XiRowsOut<L>;
    fast_dif_stage_rows<P, 0, NP, NT, true, false, 1, PITCH, GI, GO>(buf, tw, gin, gout);
    __syncthreads();
    if constexpr (P::NST == 3) {
        fast_dif_stage_rows<P, 1, NP, NT, false, false, 1, PITCH, GI, GO>(buf, tw, gin, gout);
        __syncthreads();
        fast_dif_stage_rows<P, 2, NP, NT, false, true, 1, PITCH, GI, GO>(buf, tw, gin, gout);
    } else {
        fast_dif_stage_rows<P, 1, NP, NT, false, true, 1, PITCH, GI, GO>(buf, tw, gin, gout);
    }
}

// ---- fused x + y forward over one z plane --------------------------------------
// For a grid whose x and y lengths are both L (a compile-time plan), one CTA
// transforms a whole z plane: the x transforms of its GMF row pairs and the y
// transforms of the resulting half spectra, in one shared-memory plane of
// L rows x H = L/2 + 1 columns, writing only the y spectrum B[z][ky][kx] (the
// layout of the y-forward pass) to HBM.  The x spectrum never leaves the SM.
//  - x lines: line p (rows 2p, 2p+1) lives line-major in plane rows 2p and
//    2p + 1 (2H = L + 2 >= L positions); DIF stages with consecutive threads on
//    consecutive butterflies of a line; the first reads the int64 rows from HBM;
//  - separation of the two real rows, one warp per line: it reads the line's
//    digit-reversed Z_k and Z_{L-k} into registers, then writes A_k to row 2p
//    and B_k to row 2p + 1 (column k);
//  - y: DIF stages over the H columns (element-major, consecutive threads on
//    consecutive columns), the last writing natural ky to HBM.
// The plane's x lines from the mass field (rows 2p, 2p + 1 packed as one
// complex line p, line storage LS): one thread per pair of x positions of a
// row pair, with 16-byte loads of both rows (consecutive threads on
// consecutive positions) and one 16-byte shared store of the two complex
// values; converted exactly (hardware int64 -> float rounding, power-of-two
// scale).  Positions G0 .. L-1 and the row G1 of an odd G1 are zero.  LS is
// even (2 (L/2 + 1)), so the stores are 16-byte aligned; with an odd G0 the
// last pair writes position G0 (a zero), which lies inside the line storage
// (LS >= L + 1) and is read by no x stage when G0 = L.
template <int L, int NT, int LS>
__device__ __forceinline__ void xy_load_plane(float2* buf, const int64_t* __restrict__ in, int G0, int G1, int nl,
                                              float scale) {
    const int half = (G0 + 1) / 2;   // position pairs per row
    const bool vec = !(G0 & 1) && !(reinterpret_cast<size_t>(in) & 15);
    const int items = nl * half;
#pragma unroll 4
    for (int i = threadIdx.x; i < items; i += NT) {
        const int p = i / half, x = 2 * (i - p * half);
        const bool odd_row = 2 * p + 1 < G1;
        const int64_t* r0 = in + (long long)(2 * p) * G0 + x;
        long long a0, a1, b0 = 0, b1 = 0;
        if (vec) {
            const longlong2 u = *reinterpret_cast<const longlong2*>(r0);
            a0 = u.x;
            a1 = u.y;
            if (odd_row) {
                const longlong2 w = *reinterpret_cast<const longlong2*>(r0 + G0);
                b0 = w.x;
                b1 = w.y;
            }
        } else {
            const bool x1 = x + 1 < G0;
            a0 = r0[0];
            a1 = x1 ? r0[1] : 0;
            if (odd_row) {
                b0 = r0[G0];
                b1 = x1 ? r0[G0 + 1] : 0;
            }
        }
        *reinterpret_cast<float4*>(buf + p * LS + x) =
            make_float4(fixed_to_real<float>(a0, scale), fixed_to_real<float>(b0, scale),
                        fixed_to_real<float>(a1, scale), fixed_to_real<float>(b1, scale));
    }
    const int pad = L - 2 * half;
    for (int t = threadIdx.x; t < nl * pad; t += NT) {
        const int p = t / pad;
        buf[p * LS + 2 * half + (t - p * pad)] = make_float2(0.f, 0.f);
    }
}
template <int L> struct XyOut {
    float2* __restrict__ p;          // B row ky = 0 of this plane, column 0
    int Hx;
    __device__ __forceinline__ void st(int col, int ky, float2 v) const { p[ky * Hx + col] = v; }
};

// one DIF stage of the x lines (line-major, line storage LS complex apart,
// butterflies on consecutive threads); nl lines (runtime)
template <class P, int S_, int NT, bool IN_G, int LS, class GIN>
__device__ __forceinline__ void xy_x_stage(float2* buf, const float2* __restrict__ tw, const GIN& gin, int nl) {
    constexpr int R = P::radix(S_), S = P::inner(S_), L = P::L;
    constexpr int NB = L / R;
    constexpr int TWS = L / (R * S);
    const int items = NB * nl;
#pragma unroll 1
    for (int i = threadIdx.x; i < items; i += NT) {
        const int line = i / NB, b = i - line * NB;
        const int hi = b / S, lo = b - hi * S;
        const int base = hi * R * S + lo;
        float2* lb = buf + line * LS;
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (IN_G) v[k] = gin.ld(line, base + k * S);
            else v[k] = lb[base + k * S];
        }
        FastDft<-1, R>::run(v);
        if constexpr (S > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = mul<float>(v[k], tw[lo * k * TWS]);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) lb[base + k * S] = v[k];
    }
}

// one DIF stage of the y columns (element-major, H columns, columns on
// consecutive threads)
template <class P, int S_, int NT, bool OUT_G, class GOUT>
__device__ __forceinline__ void xy_y_stage(float2* buf, const float2* __restrict__ tw, const GOUT& gout) {
    constexpr int R = P::radix(S_), S = P::inner(S_), L = P::L, H = L / 2 + 1;
    constexpr int NB = L / R, ITEMS = NB * H, TRIPS = (ITEMS + NT - 1) / NT;
    constexpr int TWS = L / (R * S);
#pragma unroll 1
    for (int it = 0; it < TRIPS; ++it) {
        const int i = threadIdx.x + it * NT;
        if (ITEMS % NT != 0 && i >= ITEMS) break;
        const int col = i % H, b = i / H;
        const int hi = b / S, lo = b - hi * S;
        const int base = hi * R * S + lo;
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = buf[(base + k * S) * H + col];
        FastDft<-1, R>::run(v);
        if constexpr (S > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = mul<float>(v[k], tw[lo * k * TWS]);
        }
        static_assert(!OUT_G || S == 1, "global output only from the last stage");
        const int nat0 = OUT_G ? P::natural(base) : 0;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (OUT_G) gout.st(col, nat0 + k * P::last_weight(), v[k]);
            else buf[(base + k * S) * H + col] = v[k];
        }
    }
}

template <class P, int NT>
__global__ void __launch_bounds__(NT, 2) k_xy_fast(const GridDev* __restrict__ grids, const Chunk* __restrict__ chunks,
                                                   const int64_t* const* __restrict__ gmf,
                                                   const float2* __restrict__ tw_arena, float2* __restrict__ wsB,
                                                   int F) {
    constexpr int L = P::L, H = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_fast[];
    float2* buf = reinterpret_cast<float2*>(smem_fast);   // L x H
    float2* tw = buf + L * H;
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    const int z = ch.tile;
    const int G0 = g.G[0], G1 = g.G[1];
    const int nl = (G1 + 1) / 2;
    for (int t = threadIdx.x; t < L; t += NT) tw[t] = tw_arena[g.fx.tw_off + t];
    // rows 2 nl .. L-1 are the y transform's zero padding
    for (int t = threadIdx.x + 2 * nl * H; t < L * H; t += NT) buf[t] = make_float2(0.f, 0.f);
    xy_load_plane<L, NT, 2 * H>(buf, gmf[ch.grid] + (long long)z * G1 * G0, G0, G1, nl, pow2_neg<float>(F));
    __syncthreads();   // twiddles and the x lines
    const NoIO none;
    xy_x_stage<P, 0, NT, false, 2 * H>(buf, tw, none, nl);
    __syncthreads();
    xy_x_stage<P, 1, NT, false, 2 * H>(buf, tw, none, nl);
    if constexpr (P::NST == 3) {
        __syncthreads();
        xy_x_stage<P, 2, NT, false, 2 * H>(buf, tw, none, nl);
    }
    __syncthreads();
    // separation, one warp per line (its storage is touched by no other warp)
    {
        constexpr int KR = (H + 31) / 32;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int p = warp; p < nl; p += NT / 32) {
            float2* lb = buf + p * 2 * H;
            float2 za[KR], zb[KR];
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int k = lane + 32 * r;
                if (k < H) {
                    za[r] = lb[P::position(k)];
                    zb[r] = lb[P::position(k == 0 ? 0 : L - k)];
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int k = lane + 32 * r;
                if (k < H) {
                    const float2 zz = za[r], zm = zb[r];
                    lb[k] = make_float2(0.5f * (zz.x + zm.x), 0.5f * (zz.y - zm.y));
                    // row G1 of an odd G1 is zero padding, exactly
                    lb[H + k] = 2 * p + 1 < G1 ? make_float2(0.5f * (zz.y + zm.y), 0.5f * (zm.x - zz.x))
                                               : make_float2(0.f, 0.f);
                }
            }
        }
    }
    __syncthreads();
    XyOut<L> gout;
    gout.p = wsB + (g.wsB + (long long)z * L * g.Hx);
    gout.Hx = g.Hx;
    xy_y_stage<P, 0, NT, false>(buf, tw, none);
    __syncthreads();
    if constexpr (P::NST == 3) {
        xy_y_stage<P, 1, NT, false>(buf, tw, none);
        __syncthreads();
        xy_y_stage<P, 2, NT, true>(buf, tw, gout);
    } else {
        xy_y_stage<P, 1, NT, true>(buf, tw, gout);
    }
}

// ---- fused y + x inverse over one window plane ------------------------------------
// The inverse of k_xy_fast's pair, for grids with M0 = M1 = L: one CTA takes
// the z pass's output plane A[zw][ky][kx] (L x H), runs the y inverse over its
// H columns and the C2R x inverse of its window row pairs in the same shared
// plane, and writes only the window phi_short[zw][yw][xw] to HBM.
//  - y: decimation-in-frequency inverse stages (conjugate twiddles) over the
//    columns, the first reading natural ky from HBM; the rows end in
//    digit-reversed order: natural row y sits at row position(y);
//  - x lines: window rows 2p, 2p+1 are natural rows ya, yb at plane rows
//    ra = position(ya), rb = position(yb); line p's element e lives at
//    (ra, e) for e < H and at (rb, e - H) beyond; one warp per line builds it
//    in place, Z_k = A_k + i B_k and Z_{L-k} = conj A_k + i conj B_k;
//  - x: decimation-in-frequency inverse stages on the lines (butterflies on
//    consecutive threads), the last writing the window cells of rows 2p and
//    2p + 1 times 1/(M0 M1 M2).
template <int L> struct YxIn {
    const float2* __restrict__ p;    // A row ky = 0 of this plane, column 0
    int Hx;
    __device__ __forceinline__ float2 ld(int col, int ky) const { return p[ky * Hx + col]; }
};

// one DIF stage of the y columns with DIR and an optional HBM input
template <class P, int S_, int NT, bool IN_G, int DIR, class GIN>
__device__ __forceinline__ void yx_y_stage(float2* buf, const float2* __restrict__ tw, const GIN& gin) {
    constexpr int R = P::radix(S_), S = P::inner(S_), L = P::L, H = L / 2 + 1;
    constexpr int NB = L / R, ITEMS = NB * H, TRIPS = (ITEMS + NT - 1) / NT;
    constexpr int TWS = L / (R * S);
#pragma unroll 1
    for (int it = 0; it < TRIPS; ++it) {
        const int i = threadIdx.x + it * NT;
        if (ITEMS % NT != 0 && i >= ITEMS) break;
        const int col = i % H, b = i / H;
        const int hi = b / S, lo = b - hi * S;
        const int base = hi * R * S + lo;
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if constexpr (IN_G) v[k] = gin.ld(col, base + k * S);
            else v[k] = buf[(base + k * S) * H + col];
        }
        FastDft<DIR, R>::run(v);
        if constexpr (S > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = mul<float>(v[k], twid<float, DIR>(tw, lo * k * TWS));
        }
#pragma unroll
        for (int k = 0; k < R; ++k) buf[(base + k * S) * H + col] = v[k];
    }
}

// the plane rows of window row pair p (natural rows (s0 + 2p) mod L and the next)
template <class P>
__device__ __forceinline__ void yx_rows(int p, int s0, int& ra, int& rb) {
    constexpr int L = P::L;
    int ya = s0 + 2 * p;
    while (ya >= L) ya -= L;
    int yb = ya + 1;
    if (yb >= L) yb -= L;
    ra = P::position(ya);
    rb = P::position(yb);
}

// one DIF inverse stage of the x lines (split rows ra | rb, butterflies on
// consecutive threads); the last stage writes the window
template <class P, int S_, int NT, bool OUT_G>
__device__ __forceinline__ void yx_x_stage(float2* buf, const float2* __restrict__ tw, int nl, int s0y, int s0x,
                                           float* __restrict__ out, int W0, int W1, float norm) {
    constexpr int R = P::radix(S_), S = P::inner(S_), L = P::L, H = L / 2 + 1;
    constexpr int NB = L / R;
    constexpr int TWS = L / (R * S);
    const int items = NB * nl;
#pragma unroll 1
    for (int i = threadIdx.x; i < items; i += NT) {
        const int line = i / NB, b = i - line * NB;
        const int hi = b / S, lo = b - hi * S;
        const int base = hi * R * S + lo;
        int ra, rb;
        yx_rows<P>(line, s0y, ra, rb);
        float2 v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int e = base + k * S;
            v[k] = e < H ? buf[ra * H + e] : buf[rb * H + e - H];
        }
        FastDft<1, R>::run(v);
        if constexpr (S > 1) {
#pragma unroll
            for (int k = 1; k < R; ++k) v[k] = mul<float>(v[k], twid<float, 1>(tw, lo * k * TWS));
        }
        if constexpr (OUT_G) {
            static_assert(S == 1, "window output only from the last stage");
            float* r0 = out + (long long)(2 * line) * W0;
            const bool has1 = 2 * line + 1 < W1;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                int w = P::natural(base) + k * P::last_weight() - s0x;
                if (w < 0) w += L;
                for (; w < W0; w += L) {
                    r0[w] = v[k].x * norm;
                    if (has1) r0[W0 + w] = v[k].y * norm;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const int e = base + k * S;
                if (e < H) buf[ra * H + e] = v[k];
                else buf[rb * H + e - H] = v[k];
            }
        }
    }
}

template <class P, int NT>
__global__ void __launch_bounds__(NT, 2) k_yx_fast(const GridDev* __restrict__ grids, const Chunk* __restrict__ chunks,
                                                   const float2* __restrict__ tw_arena,
                                                   const float2* __restrict__ wsA, void* const* __restrict__ phis,
                                                   int comp) {
    constexpr int L = P::L, H = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_fast[];
    float2* buf = reinterpret_cast<float2*>(smem_fast);   // L x H
    float2* tw = buf + L * H;
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    const int zw = ch.tile;
    const int W0 = g.W[0], W1 = g.W[1];
    const int nl = (W1 + 1) / 2;
    for (int t = threadIdx.x; t < L; t += NT) tw[t] = tw_arena[g.fx.tw_off + t];
    YxIn<L> gin;
    gin.p = wsA + (g.wsA + (long long)zw * L * g.Hx);
    gin.Hx = g.Hx;
    __syncthreads();   // twiddles
    yx_y_stage<P, 0, NT, true, 1>(buf, tw, gin);
    __syncthreads();
    yx_y_stage<P, 1, NT, false, 1>(buf, tw, gin);
    __syncthreads();
    if constexpr (P::NST == 3) {
        yx_y_stage<P, 2, NT, false, 1>(buf, tw, gin);
        __syncthreads();
    }
    // the window's row pairs as complex lines, one warp per line
    const int s0y = g.s0[1], s0x = g.s0[0];
    {
        constexpr int KR = (H + 31) / 32;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int p = warp; p < nl; p += NT / 32) {
            int ra, rb;
            yx_rows<P>(p, s0y, ra, rb);
            const bool has1 = 2 * p + 1 < W1;
            float2 av[KR], bv[KR];
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int k = lane + 32 * r;
                if (k < H) {
                    av[r] = buf[ra * H + k];
                    bv[r] = has1 ? buf[rb * H + k] : make_float2(0.f, 0.f);
                }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < KR; ++r) {
                const int k = lane + 32 * r;
                if (k < H) {
                    const float2 a = av[r], bb = bv[r];
                    buf[ra * H + k] = make_float2(a.x - bb.y, a.y + bb.x);            // element k
                    if (k > 0 && L - k >= H)                                         // element L - k
                        buf[rb * H + (L - k - H)] = make_float2(a.x + bb.y, bb.x - a.y);
                }
            }
        }
    }
    __syncthreads();
    float* out = reinterpret_cast<float*>(phis[ch.grid]) + (long long)comp * g.W[0] * g.W[1] * g.W[2] +
                 (long long)zw * W1 * W0;
    const float norm = (float)g.inv_m3;
    yx_x_stage<P, 0, NT, false>(buf, tw, nl, s0y, s0x, out, W0, W1, norm);
    __syncthreads();
    if constexpr (P::NST == 3) {
        yx_x_stage<P, 1, NT, false>(buf, tw, nl, s0y, s0x, out, W0, W1, norm);
        __syncthreads();
        yx_x_stage<P, 2, NT, true>(buf, tw, nl, s0y, s0x, out, W0, W1, norm);
    } else {
        yx_x_stage<P, 1, NT, true>(buf, tw, nl, s0y, s0x, out, W0, W1, norm);
    }
}

}  // namespace
}  // namespace apm

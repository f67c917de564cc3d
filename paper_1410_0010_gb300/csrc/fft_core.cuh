// fft_core.cuh -- batched 3-D FFT convolution of every grid of a level (Sec. 2.2,
// Eq. PoissonFourier): the zero-padded GMF of each grid is transformed on its
// M0 x M1 x M2 grid, multiplied by the Green's table and transformed back; only
// the window of cells [-2, N+2) of the result is written.
//
// Five passes, each one CTA per batch of lines, each line transformed entirely
// in shared memory by mixed-radix Stockham stages (radices 2-8, and on the FP32
// path the composites 6, 9, 10, 12, 14, 15, 16 done in registers; ping-pong
// between two shared-memory buffers, twiddles staged in shared memory).  A CTA
// holds a power-of-two number of lines, laid out element-major (line index
// fastest), so consecutive threads take consecutive lines and no integer
// division is left in the butterfly loops:
//   xf : GMF rows (int64 -> FP64 mass -> T), two real rows per complex line,
//        R2C along x                                   -> A[z][y][kx]   (y < G1, z < G2)
//   yf : columns along y, zero-padded G1 -> M1         -> B[z][ky][kx]  (z < G2)
//   z  : columns along z, zero-padded G2 -> M2, times the table, inverse,
//        window of W2 planes                           -> A[zw][ky][kx]
//   yi : columns along y, inverse, window of W1 rows   -> B[zw][yw][kx]
//   xi : rows, C2R (two real rows per complex line), window of W0 cells,
//        scaled by 1/(M0 M1 M2)                        -> phi_short[zw][yw][xw]
// Zero-padded inputs are never read and outputs outside the window never
// written.  Lines of the y/z passes are tiles of consecutive kx (coalesced).
#pragma once
#include <type_traits>
#include <utility>

#include "apm_internal.cuh"

// The pass kernels and their building blocks, as templates; k_fft_x.cu and
// k_fft_col.cu (once per precision and column pass) instantiate them, so the
// instantiations compile in parallel.
namespace apm {
namespace {

template <typename T> using C = typename Cplx<T>::type;

// minimum resident CTAs per SM the pass kernels are compiled for
#ifndef APM_FFT_MIN_CTAS
#define APM_FFT_MIN_CTAS 4
#endif
template <typename T> struct MinCtas { static constexpr int value = APM_FFT_MIN_CTAS; };
template <> struct MinCtas<double> { static constexpr int value = 1; };

template <typename T> __device__ __forceinline__ C<T> mk(T a, T b) { C<T> r; r.x = a; r.y = b; return r; }
template <typename T> __device__ __forceinline__ C<T> add(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> sub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> mul(C<T> a, C<T> b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by exp(DIR * i pi / 2) = DIR * i
template <typename T, int DIR> __device__ __forceinline__ C<T> rot90(C<T> a) {
    return DIR < 0 ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
}

// exp(DIR 2 pi i t / L) from the table of exp(-2 pi i t / L)
template <typename T, int DIR> __device__ __forceinline__ C<T> twid(const C<T>* tw, int t) {
    C<T> w = tw[t];
    if (DIR > 0) w.y = -w.y;
    return w;
}

// ---- roots of unity as compile-time constants --------------------------------
// cos and sin of a reduced angle |x| <= pi/4 by their Taylor series (terms to
// x^27: the truncation error is below 1e-30), evaluated by the compiler.
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double ct_sin(double x) {
    double term = x, sum = x;
    for (int n = 1; n <= 13; ++n) {
        term *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double ct_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int n = 1; n <= 13; ++n) {
        term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
// cos / sin of 2 pi m / R: the quadrant q = floor(4m/R) and the remainder
// r = 4m - qR (in units of pi/(2R)) are integers, so multiples of pi/2 are exact
// and the series only sees angles up to pi/4.
constexpr double ct_cs(int m, int R, bool want_sin) {
    const int u = ((m % R) + R) % R;
    const int q = (4 * u) / R, r = 4 * u - q * R;
    double c = 1.0, s = 0.0;                 // of phi = r pi / (2R), 0 <= phi < pi/2
    if (r != 0) {
        if (2 * r <= R) {
            c = ct_cos(r * kPi / (2.0 * R));
            s = ct_sin(r * kPi / (2.0 * R));
        } else {
            c = ct_sin((R - r) * kPi / (2.0 * R));
            s = ct_cos((R - r) * kPi / (2.0 * R));
        }
    }
    double cc = c, ss = s;                   // rotate by q quarter turns
    if (q == 1) { cc = -s; ss = c; }
    if (q == 2) { cc = -c; ss = -s; }
    if (q == 3) { cc = s; ss = -c; }
    return want_sin ? ss : cc;
}
// v times exp(DIR 2 pi i m / R); quarter turns are exact rotations
template <typename T, int DIR, int M, int R> __device__ __forceinline__ C<T> mul_root(C<T> v) {
    constexpr int u = ((M % R) + R) % R;
    constexpr int quarter = (4 * u) % R == 0 ? (4 * u) / R : -1;
    if constexpr (quarter == 0) {
        return v;
    } else if constexpr (quarter == 2) {
        return mk<T>(-v.x, -v.y);
    } else if constexpr (quarter == 1 || quarter == 3) {
        // (DIR i)^quarter: i when DIR quarter = 1 mod 4, -i when 3 mod 4
        constexpr int turn = (((DIR * quarter) % 4) + 4) % 4;
        if constexpr (turn == 1) return mk<T>(-v.y, v.x);
        else return mk<T>(v.y, -v.x);
    } else {
        constexpr T re = (T)ct_cs(M, R, false);
        constexpr T im = (T)(DIR * ct_cs(M, R, true));
        return mk<T>(v.x * re - v.y * im, v.x * im + v.y * re);
    }
}

// compile-time loop: f(std::integral_constant<int, 0>) ... f(<N-1>)
template <typename F, int... I>
__device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F> __device__ __forceinline__ void sfor(F&& f) {
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// In-register DFT of size R: X_q = sum_r v_r exp(DIR 2 pi i q r / R).
template <typename T, int DIR, int R> struct Dft;

template <typename T, int DIR> struct Dft<T, DIR, 2> {
    __device__ static void run(C<T>* v) {
        C<T> a = v[0], b = v[1];
        v[0] = add<T>(a, b);
        v[1] = sub<T>(a, b);
    }
};

template <typename T, int DIR> struct Dft<T, DIR, 4> {
    __device__ static void run(C<T>* v) {
        C<T> t0 = add<T>(v[0], v[2]), t1 = sub<T>(v[0], v[2]);
        C<T> t2 = add<T>(v[1], v[3]), t3 = rot90<T, DIR>(sub<T>(v[1], v[3]));
        v[0] = add<T>(t0, t2);
        v[2] = sub<T>(t0, t2);
        v[1] = add<T>(t1, t3);
        v[3] = sub<T>(t1, t3);
    }
};

template <typename T, int DIR> struct Dft<T, DIR, 8> {
    __device__ static void run(C<T>* v) {
        C<T> e[4] = {v[0], v[2], v[4], v[6]};
        C<T> o[4] = {v[1], v[3], v[5], v[7]};
        Dft<T, DIR, 4>::run(e);
        Dft<T, DIR, 4>::run(o);
        const T h = (T)0.70710678118654752440084436210484903928;
        // o_q * exp(DIR 2 pi i q / 8)
        C<T> o1 = mk<T>(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
        C<T> o2 = rot90<T, DIR>(o[2]);
        C<T> o3 = mk<T>(-h * (o[3].x + DIR * o[3].y), h * (DIR * o[3].x - o[3].y));
        v[0] = add<T>(e[0], o[0]);
        v[4] = sub<T>(e[0], o[0]);
        v[1] = add<T>(e[1], o1);
        v[5] = sub<T>(e[1], o1);
        v[2] = add<T>(e[2], o2);
        v[6] = sub<T>(e[2], o2);
        v[3] = add<T>(e[3], o3);
        v[7] = sub<T>(e[3], o3);
    }
};

// odd prime R (3, 5, 7): with a_k = v_k + v_{R-k}, b_k = v_k - v_{R-k}
// (k = 1 .. (R-1)/2),
//   X_0     = v_0 + sum_k a_k
//   X_q     = v_0 + sum_k cos(2 pi qk/R) a_k + DIR i sum_k sin(2 pi qk/R) b_k
//   X_{R-q} = the same with -DIR i,
// every cosine and sine a compile-time constant.
template <typename T, int DIR, int R> struct Dft {
    __device__ static void run(C<T>* v) {
        constexpr int H = (R - 1) / 2;
        C<T> a[H], b[H];
        const C<T> x0 = v[0];
        C<T> s0 = x0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            a[k - 1] = add<T>(v[k], v[R - k]);
            b[k - 1] = sub<T>(v[k], v[R - k]);
            s0 = add<T>(s0, a[k - 1]);
        }
        sfor<H>([&](auto qi) {
            constexpr int q = decltype(qi)::value + 1;
            C<T> re = x0, im = mk<T>(0, 0);
            sfor<H>([&](auto ki) {
                constexpr int k = decltype(ki)::value + 1;
                constexpr T c = (T)ct_cs(q * k, R, false);
                constexpr T sn = (T)ct_cs(q * k, R, true);
                re.x += c * a[k - 1].x;
                re.y += c * a[k - 1].y;
                im.x += sn * b[k - 1].x;
                im.y += sn * b[k - 1].y;
            });
            // DIR i im
            const C<T> r = DIR > 0 ? mk<T>(-im.y, im.x) : mk<T>(im.y, -im.x);
            v[q] = add<T>(re, r);
            v[R - q] = sub<T>(re, r);
        });
        v[0] = s0;
    }
};

// Composite radix R = R1 R2 in registers (Cooley-Tukey inside the butterfly):
// with n = R2 n1 + n2 and k = k1 + R1 k2,
//   X[k1 + R1 k2] = sum_n2 w_R2^(n2 k2) w_R^(n2 k1) sum_n1 v[R2 n1 + n2] w_R1^(n1 k1),
// w_m = exp(DIR 2 pi i / m); every w_R^(n2 k1) is a compile-time constant.
template <typename T, int DIR, int R1, int R2>
struct DftC {
    __device__ static void run(C<T>* v) {
        constexpr int R = R1 * R2;
        sfor<R2>([&](auto n2i) {
            constexpr int n2 = decltype(n2i)::value;
            C<T> t[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + n2];
            Dft<T, DIR, R1>::run(t);
            sfor<R1>([&](auto k1i) {
                constexpr int k1 = decltype(k1i)::value;
                v[R2 * k1 + n2] = mul_root<T, DIR, n2 * k1, R>(t[k1]);
            });
        });
        C<T> out[R];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            C<T> t[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) t[n2] = v[R2 * k1 + n2];
            Dft<T, DIR, R2>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) out[k1 + R1 * k2] = t[k2];
        }
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = out[q];
    }
};

// One Stockham stage of radix R over nl = 2^lg lines of length L, element i of
// line l at [i*es + l], from src to dst; Ns = product of the radices already
// applied.  Butterfly j reads elements j + r L/R, twiddles them by
// exp(DIR 2 pi i (j mod Ns) r / (Ns R)), and writes elements
// (j / Ns) Ns R + (j mod Ns) + r Ns: natural order after the last stage.
// Thread t owns line t mod nl and butterflies j = t / nl + m (threads / nl);
// j / Ns and j mod Ns are stepped incrementally (the first ones by a
// multiply-high with magic = ceil(2^32 / Ns), exact for j < 2^21).
__device__ __forceinline__ int div_small(int n, int d, unsigned magic) {
    return d == 1 ? n : (int)__umulhi((unsigned)n, magic);
}

template <typename T, int DIR, int R1, int R2, int NT>
__device__ void stage(const C<T>* __restrict__ src, C<T>* __restrict__ dst, int L, int Ns, int step,
                      unsigned magic, int lg, int es, const C<T>* __restrict__ tw) {
    constexpr int R = R1 * R2;
    const int nb = L / R;
    const int line = threadIdx.x & ((1 << lg) - 1);
    const int jstep = NT >> lg;
    int j = threadIdx.x >> lg;
    if (j < nb) {
        int k = div_small(j, Ns, magic), jm = j - k * Ns;
        const int dk = div_small(jstep, Ns, magic), djm = jstep - dk * Ns;
        for (; j < nb; j += jstep) {
            C<T> v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * es + line];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = mul<T>(v[r], twid<T, DIR>(tw, jm * r * step));
            }
            if constexpr (R2 == 1) Dft<T, DIR, R1>::run(v);
            else DftC<T, DIR, R1, R2>::run(v);
            const int idx = k * Ns * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[(idx + r * Ns) * es + line] = v[r];
            jm += djm;
            k += dk;
            if (jm >= Ns) {
                jm -= Ns;
                ++k;
            }
        }
    }
    __syncthreads();
}

// composite stage radices (FP32 plans only)
template <typename T, int DIR, int NT>
__device__ __forceinline__ void stage_composite(int R, const C<T>* a, C<T>* b, int L, int Ns, int step,
                                                unsigned magic, int lg, int es, const C<T>* tw) {
    switch (R) {
        case 6: stage<T, DIR, 3, 2, NT>(a, b, L, Ns, step, magic, lg, es, tw); break;
        case 9: stage<T, DIR, 3, 3, NT>(a, b, L, Ns, step, magic, lg, es, tw); break;
        case 10: stage<T, DIR, 5, 2, NT>(a, b, L, Ns, step, magic, lg, es, tw); break;
        case 12: stage<T, DIR, 3, 4, NT>(a, b, L, Ns, step, magic, lg, es, tw); break;
        case 14: stage<T, DIR, 7, 2, NT>(a, b, L, Ns, step, magic, lg, es, tw); break;
        case 15: stage<T, DIR, 5, 3, NT>(a, b, L, Ns, step, magic, lg, es, tw); break;
        default: stage<T, DIR, 4, 4, NT>(a, b, L, Ns, step, magic, lg, es, tw); break;   // 16
    }
}

// Full transform of the lines in `a` (`b`: scratch of the same size, tw: the
// length-L twiddles in shared memory); returns the buffer holding the result.
// Stage radices 2..8 directly; on the FP32 path also the composites of
// fft_plan (apm_internal.cuh), computed in registers as R1 x R2.
template <typename T, int DIR, int NT>
__device__ C<T>* fft_lines(C<T>* a, C<T>* b, const FftPlan1D& pl, int lg, int es, const C<T>* tw) {
    const int L = pl.L;
    for (int st = 0; st < pl.nst; ++st) {
        const int R = pl.radix[st], Ns = pl.ns[st], step = pl.step[st];
        const unsigned mg = pl.magic[st];
        switch (R) {
            case 2: stage<T, DIR, 2, 1, NT>(a, b, L, Ns, step, mg, lg, es, tw); break;
            case 3: stage<T, DIR, 3, 1, NT>(a, b, L, Ns, step, mg, lg, es, tw); break;
            case 4: stage<T, DIR, 4, 1, NT>(a, b, L, Ns, step, mg, lg, es, tw); break;
            case 5: stage<T, DIR, 5, 1, NT>(a, b, L, Ns, step, mg, lg, es, tw); break;
            case 7: stage<T, DIR, 7, 1, NT>(a, b, L, Ns, step, mg, lg, es, tw); break;
            case 8: stage<T, DIR, 8, 1, NT>(a, b, L, Ns, step, mg, lg, es, tw); break;
            default:
                if constexpr (sizeof(T) == 4) stage_composite<T, DIR, NT>(R, a, b, L, Ns, step, mg, lg, es, tw);
                break;
        }
        C<T>* t = a;
        a = b;
        b = t;
    }
    return a;
}

template <typename T> __device__ __forceinline__ C<T>* smem_c() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<C<T>*>(smem_raw);
}

__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

// copies the twiddles exp(-2 pi i t / L), t < L, into shared memory
template <typename T, int NT>
__device__ __forceinline__ void load_twiddles(C<T>* dst, const C<T>* __restrict__ src, int L) {
    for (int t = threadIdx.x; t < L; t += NT) dst[t] = src[t];
}

// Correctly rounded conversion of a fixed-point cell mass q * 2^-F to T:
// q rounded to nearest-even in T (the hardware int64 conversion), then scaled
// by scale = 2^-F, which is exact.  For T = float this equals the FP64
// conversion (double)q * 2^-F rounded to float whenever |q| < 2^53.
template <typename T> __device__ __forceinline__ T fixed_to_real(long long q, T scale);
template <> __device__ __forceinline__ double fixed_to_real<double>(long long q, double scale) {
    return __ll2double_rn(q) * scale;
}
template <> __device__ __forceinline__ float fixed_to_real<float>(long long q, float scale) {
    return __ll2float_rn(q) * scale;
}

// 2^-F in T, 1 <= F <= 62
template <typename T> __device__ __forceinline__ T pow2_neg(int F);
template <> __device__ __forceinline__ float pow2_neg<float>(int F) { return __int_as_float((127 - F) << 23); }
template <> __device__ __forceinline__ double pow2_neg<double>(int F) {
    return __longlong_as_double((long long)(1023 - F) << 52);
}

// ---- column passes -----------------------------------------------------------
// AX = 1 (y) or 2 (z).  MODE 0: forward only; 1: forward, table, inverse; 2: inverse only.
//   yf (AX 1, MODE 0): in A[z][y][kx] (y < G1), out B[z][ky][kx]
//   z  (AX 2, MODE 1): in B[z][ky][kx] (z < G2), out A[zw][ky][kx]
//   yi (AX 1, MODE 2): in A[zw][ky][kx],         out B[zw][yw][kx]
// A CTA holds tx consecutive kx columns (its lines).  The first stage of a
// transform reads its butterfly inputs straight from global memory (a warp
// reads consecutive kx: coalesced) and the last stage writes straight to
// global memory, so a transform of S stages makes S - 1 trips through shared
// memory.  The z pass runs the forward transform with the plan of M2 and the
// inverse with the reversed plan, whose first radix is the forward's last:
// the forward's last butterfly, the table multiply and the inverse's first
// butterfly act on the same elements in registers.
// smem: two buffers of L x tx (element-major, line fastest), twiddles (L)

// element i of this thread's line in a shared-memory buffer
template <typename T> struct SmemIO {
    C<T>* buf;
    int tx, line;
    __device__ C<T> ld(int i) const { return buf[i * tx + line]; }
    __device__ void st(int i, C<T> v) const { buf[i * tx + line] = v; }
};
// element i of this thread's global line: in[i stride] for i < n (zero beyond:
// the padding), nothing for a column outside [0, Hx)
// (i stride < 2^31: lines hold at most 1024 elements and strides are below
// 1024 x 513 elements, so the offsets stay 32-bit)
template <typename T> struct GlobalIn {
    const C<T>* __restrict__ p;
    int stride;
    int n;
    bool live;
    __device__ C<T> ld(int i) const { return (live && i < n) ? p[i * stride] : mk<T>(0, 0); }
};
// output element i of this thread's global line: window index w = (i - s0) mod L,
// written as out[w stride] when w < n, and again at w + L when that is inside
// the window too (a periodic root's window N + 4 exceeds M = N)
template <typename T> struct GlobalOut {
    C<T>* __restrict__ p;
    int stride;
    int n, s0, L;
    bool live;
    __device__ void st(int i, C<T> v) const {
        int w = i - s0;
        if (w < 0) w += L;
        if (!live) return;
        if (w < n) p[w * stride] = v;
        if (w + L < n) p[(w + L) * stride] = v;
    }
};

// One Stockham stage of radix R = R1 R2 (see stage()) with the butterfly
// inputs from `in` and the outputs to `out`; no barrier.
template <typename T, int DIR, int R1, int R2, int NT, class IN, class OUT>
__device__ __forceinline__ void stage_io(int L, int Ns, int step, unsigned magic, int lg,
                                         const C<T>* __restrict__ tw, const IN& in, const OUT& out) {
    constexpr int R = R1 * R2;
    const int nb = L / R;
    const int jstep = NT >> lg;
    int j = threadIdx.x >> lg;
    if (j >= nb) return;
    int k = div_small(j, Ns, magic), jm = j - k * Ns;
    const int dk = div_small(jstep, Ns, magic), djm = jstep - dk * Ns;
    for (; j < nb; j += jstep) {
        C<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in.ld(j + r * nb);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = mul<T>(v[r], twid<T, DIR>(tw, jm * r * step));
        }
        if constexpr (R2 == 1) Dft<T, DIR, R1>::run(v);
        else DftC<T, DIR, R1, R2>::run(v);
        const int idx = k * Ns * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) out.st(idx + r * Ns, v[r]);
        jm += djm;
        k += dk;
        if (jm >= Ns) {
            jm -= Ns;
            ++k;
        }
    }
}

template <typename T, int DIR, int NT, class IN, class OUT>
__device__ void stage_any(int R, int L, int Ns, int step, unsigned magic, int lg, const C<T>* tw,
                          const IN& in, const OUT& out) {
    switch (R) {
        case 2: stage_io<T, DIR, 2, 1, NT>(L, Ns, step, magic, lg, tw, in, out); break;
        case 3: stage_io<T, DIR, 3, 1, NT>(L, Ns, step, magic, lg, tw, in, out); break;
        case 4: stage_io<T, DIR, 4, 1, NT>(L, Ns, step, magic, lg, tw, in, out); break;
        case 5: stage_io<T, DIR, 5, 1, NT>(L, Ns, step, magic, lg, tw, in, out); break;
        case 7: stage_io<T, DIR, 7, 1, NT>(L, Ns, step, magic, lg, tw, in, out); break;
        case 8: stage_io<T, DIR, 8, 1, NT>(L, Ns, step, magic, lg, tw, in, out); break;
        default:
            if constexpr (sizeof(T) == 4) {
                switch (R) {
                    case 6: stage_io<T, DIR, 3, 2, NT>(L, Ns, step, magic, lg, tw, in, out); break;
                    case 9: stage_io<T, DIR, 3, 3, NT>(L, Ns, step, magic, lg, tw, in, out); break;
                    case 10: stage_io<T, DIR, 5, 2, NT>(L, Ns, step, magic, lg, tw, in, out); break;
                    case 12: stage_io<T, DIR, 3, 4, NT>(L, Ns, step, magic, lg, tw, in, out); break;
                    case 14: stage_io<T, DIR, 7, 2, NT>(L, Ns, step, magic, lg, tw, in, out); break;
                    case 15: stage_io<T, DIR, 5, 3, NT>(L, Ns, step, magic, lg, tw, in, out); break;
                    default: stage_io<T, DIR, 4, 4, NT>(L, Ns, step, magic, lg, tw, in, out); break;
                }
            }
            break;
    }
}

// Stages [s_first, s_last] of plan pl.  The first reads `in` (IN_SMEM: the
// shared buffer *cur), the last writes `out` (OUT_SMEM: the shared buffer
// *nxt); the stages between ping-pong through the shared buffers.  After every
// stage that wrote shared memory: a barrier, and cur / nxt swap, so on return
// *cur holds the last shared result.
template <typename T, int DIR, int NT, bool IN_SMEM, bool OUT_SMEM, class IN, class OUT>
__device__ void stages_io(const FftPlan1D& pl, int s_first, int s_last, int lg, const C<T>* tw,
                          const IN& in, const OUT& out, C<T>*& cur, C<T>*& nxt, int tx, int line) {
    const int L = pl.L;
    for (int st = s_first; st <= s_last; ++st) {
        const int R = pl.radix[st], Ns = pl.ns[st], step = pl.step[st];
        const unsigned mg = pl.magic[st];
        const bool gin = st == s_first && !IN_SMEM, gout = st == s_last && !OUT_SMEM;
        const SmemIO<T> sin{cur, tx, line}, sout{nxt, tx, line};
        if (gin) {
            if constexpr (!IN_SMEM) {
                if (gout) {
                    if constexpr (!OUT_SMEM) stage_any<T, DIR, NT>(R, L, Ns, step, mg, lg, tw, in, out);
                } else {
                    stage_any<T, DIR, NT>(R, L, Ns, step, mg, lg, tw, in, sout);
                }
            }
        } else if (gout) {
            if constexpr (!OUT_SMEM) stage_any<T, DIR, NT>(R, L, Ns, step, mg, lg, tw, sin, out);
        } else {
            stage_any<T, DIR, NT>(R, L, Ns, step, mg, lg, tw, sin, sout);
        }
        if (!gout) {
            __syncthreads();
            C<T>* t = cur;
            cur = nxt;
            nxt = t;
        }
    }
}

// The z pass's middle: the forward plan's last stage (radix R, Ns = L/R), the
// table multiply of its outputs (element j + r L/R), and the reversed plan's
// first stage (radix R, Ns = 1) on the same elements, writing j R + r.
template <typename T, int R1, int R2, int NT, class IN, class OUT, class TAB>
__device__ __forceinline__ void stage_fwd_tab_inv(int L, int step, int lg, const C<T>* __restrict__ tw,
                                                  const IN& in, const OUT& out, const TAB& tabf) {
    constexpr int R = R1 * R2;
    const int nb = L / R;
    const int jstep = NT >> lg;
    for (int j = threadIdx.x >> lg; j < nb; j += jstep) {
        C<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in.ld(j + r * nb);
        if (nb > 1) {   // Ns = nb: the twiddle of butterfly j is exp(-2 pi i j r / L)
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = mul<T>(v[r], twid<T, -1>(tw, j * r * step));
        }
        if constexpr (R2 == 1) Dft<T, -1, R1>::run(v);
        else DftC<T, -1, R1, R2>::run(v);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = tabf.apply(j + r * nb, v[r]);
        if constexpr (R2 == 1) Dft<T, 1, R1>::run(v);
        else DftC<T, 1, R1, R2>::run(v);
#pragma unroll
        for (int r = 0; r < R; ++r) out.st(j * R + r, v[r]);
    }
}

template <typename T, int NT, class IN, class OUT, class TAB>
__device__ void fwd_tab_inv_any(int R, int L, int step, int lg, const C<T>* tw, const IN& in, const OUT& out,
                                const TAB& tabf) {
    switch (R) {
        case 2: stage_fwd_tab_inv<T, 2, 1, NT>(L, step, lg, tw, in, out, tabf); break;
        case 3: stage_fwd_tab_inv<T, 3, 1, NT>(L, step, lg, tw, in, out, tabf); break;
        case 4: stage_fwd_tab_inv<T, 4, 1, NT>(L, step, lg, tw, in, out, tabf); break;
        case 5: stage_fwd_tab_inv<T, 5, 1, NT>(L, step, lg, tw, in, out, tabf); break;
        case 7: stage_fwd_tab_inv<T, 7, 1, NT>(L, step, lg, tw, in, out, tabf); break;
        case 8: stage_fwd_tab_inv<T, 8, 1, NT>(L, step, lg, tw, in, out, tabf); break;
        default:
            if constexpr (sizeof(T) == 4) {
                switch (R) {
                    case 6: stage_fwd_tab_inv<T, 3, 2, NT>(L, step, lg, tw, in, out, tabf); break;
                    case 9: stage_fwd_tab_inv<T, 3, 3, NT>(L, step, lg, tw, in, out, tabf); break;
                    case 10: stage_fwd_tab_inv<T, 5, 2, NT>(L, step, lg, tw, in, out, tabf); break;
                    case 12: stage_fwd_tab_inv<T, 3, 4, NT>(L, step, lg, tw, in, out, tabf); break;
                    case 14: stage_fwd_tab_inv<T, 7, 2, NT>(L, step, lg, tw, in, out, tabf); break;
                    case 15: stage_fwd_tab_inv<T, 5, 3, NT>(L, step, lg, tw, in, out, tabf); break;
                    default: stage_fwd_tab_inv<T, 4, 4, NT>(L, step, lg, tw, in, out, tabf); break;
                }
            }
            break;
    }
}

// table value of element kz of this thread's (ky, kx) column: T is even in
// every component, stored as an octant
template <typename T> struct TabCol {
    const T* __restrict__ p;   // at (|ky|, kx)
    int zst, L;
    __device__ T operator()(int kz) const { return p[(kz <= L / 2 ? kz : L - kz) * zst]; }
    __device__ C<T> apply(int kz, C<T> v) const {
        const T t = (*this)(kz);
        return mk<T>(v.x * t, v.y * t);
    }
};

// Spectral gradient component comp (1 x, 2 y, 3 z): v -> -i D T v with
// D = k_comp, 0 on the Nyquist mode of an even length (the table is even, the
// factor odd, so the product keeps the Hermitian symmetry of a real field).
// dline: D of the column's kx (comp 1) or ky (comp 2); dz: 2 pi / (M2 delta).
template <typename T> struct TabGrad {
    TabCol<T> tab;
    int comp;
    T dline, dz;
    __device__ C<T> apply(int kz, C<T> v) const {
        T d = dline;
        if (comp == 3) {
            const int L = tab.L;
            d = 2 * kz == L ? T(0) : dz * (T)(kz <= L / 2 ? kz : kz - L);
        }
        const T s = tab(kz) * d;
        return mk<T>(v.y * s, -v.x * s);
    }
};

template <typename T, int AX, int MODE, int NT>
__global__ void __launch_bounds__(NT, MinCtas<T>::value * (kFftThreads / NT)) k_col(const GridDev* __restrict__ grids,
                                                     const Chunk* __restrict__ chunks,
                                                     const C<T>* __restrict__ tw_arena,
                                                     const T* __restrict__ tab,
                                                     C<T>* __restrict__ wsA, C<T>* __restrict__ wsB,
                                                     int comp) {
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    const int Hx = g.Hx;
    const int tx = g.lines[AX == 2 ? kPassZ : (MODE == 0 ? kPassYf : kPassYi)];
    const int lg = ilog2(tx);
    const int other = ch.tile & ((1 << kColOtherBits) - 1);    // z (yf), ky (z), zw (yi)
    const int kx0 = (ch.tile >> kColOtherBits) << lg;
    const FftPlan1D& pl = AX == 1 ? (MODE == 0 ? g.fy : g.iy) : g.fz;
    const int L = pl.L;
    const int M1 = g.M[1];
    C<T>* cur = smem_c<T>();
    C<T>* nxt = cur + L * tx;
    C<T>* tw = nxt + L * tx;
    load_twiddles<T, NT>(tw, tw_arena + pl.tw_off, L);
    const int line = threadIdx.x & (tx - 1);
    const int kx = kx0 + line;
    const bool live = kx < Hx;

    GlobalIn<T> in;
    GlobalOut<T> out;
    in.live = out.live = live;
    out.L = L;
    if (AX == 1 && MODE == 0) {
        in.p = wsA + (g.wsA + (long long)other * g.G[1] * Hx + kx); in.stride = Hx; in.n = g.G[1];
        out.p = wsB + (g.wsB + (long long)other * M1 * Hx + kx); out.stride = Hx; out.n = M1; out.s0 = 0;
    } else if (AX == 2) {
        in.p = wsB + (g.wsB + (long long)other * Hx + kx); in.stride = M1 * Hx; in.n = g.G[2];
        out.p = wsA + (g.wsA + (long long)other * Hx + kx); out.stride = M1 * Hx;
        out.n = g.W[2]; out.s0 = g.s0[2];
    } else {
        in.p = wsA + (g.wsA + (long long)other * M1 * Hx + kx); in.stride = Hx; in.n = M1;
        out.p = wsB + (g.wsB + (long long)other * g.W[1] * Hx + kx); out.stride = Hx;
        out.n = g.W[1]; out.s0 = g.s0[1];
    }
    __syncthreads();   // twiddles
    if (MODE == 0) {
        stages_io<T, -1, NT, false, false>(pl, 0, pl.nst - 1, lg, tw, in, out, cur, nxt, tx, line);
    } else if (MODE == 2) {
        stages_io<T, 1, NT, false, false>(pl, 0, pl.nst - 1, lg, tw, in, out, cur, nxt, tx, line);
    } else {
        // phi-hat = T(kappa) rho-hat between the forward and the inverse
        // transform (MODE 1); MODE 3: -i D_comp T(kappa) rho-hat
        const FftPlan1D& ipl = g.iz;
        const int ky = other;
        const int fy = ky <= M1 / 2 ? ky : M1 - ky;
        TabCol<T> tabc;
        tabc.p = tab + (g.tab_off + (long long)fy * Hx + kx);
        tabc.zst = g.Hy2 * Hx;     // the octant table holds < 2^31 entries
        tabc.L = L;
        using Tab = typename std::conditional<MODE == 3, TabGrad<T>, TabCol<T>>::type;
        Tab tabf;
        if constexpr (MODE == 3) {
            tabf.tab = tabc;
            tabf.comp = comp;
            tabf.dz = (T)g.dk[2];
            const int M0 = g.M[0];
            const int kyc = ky <= M1 / 2 ? ky : ky - M1;
            tabf.dline = comp == 1 ? (2 * kx == M0 ? T(0) : (T)(g.dk[0] * kx))
                                   : (comp == 2 ? (2 * ky == M1 ? T(0) : (T)(g.dk[1] * kyc)) : T(0));
        } else {
            tabf = tabc;
        }
        const int n = pl.nst;
        const int R = pl.radix[n - 1];
        if (n == 1) {
            fwd_tab_inv_any<T, NT>(R, L, pl.step[0], lg, tw, in, out, tabf);
        } else {
            stages_io<T, -1, NT, false, true>(pl, 0, n - 2, lg, tw, in, out, cur, nxt, tx, line);
            fwd_tab_inv_any<T, NT>(R, L, pl.step[n - 1], lg, tw, SmemIO<T>{cur, tx, line},
                                   SmemIO<T>{nxt, tx, line}, tabf);
            __syncthreads();
            C<T>* t = cur;
            cur = nxt;
            nxt = t;
            stages_io<T, 1, NT, true, false>(ipl, 1, n - 1, lg, tw, in, out, cur, nxt, tx, line);
        }
    }
}

// ---- x passes ------------------------------------------------------------------
// A CTA holds np complex lines, each packing two real rows (2p, 2p+1) of the
// grid (two-for-one real transforms); the same thread mapping as the column
// passes (line fastest), so a warp reads 32 / np consecutive x of each of its
// rows.  smem: two buffers of M0 x (np+1) (element-major, padded), twiddles (M0)

// xi input: Z_k = A_k + i B_k, A, B the half spectra of rows 2p, 2p+1 extended
// by Hermitian symmetry (A_{M-k} = conj A_k)
template <typename T> struct XiIn {
    const C<T>* __restrict__ p;      // row 2 line of this CTA
    int Hx, M0, nr0, nr1;
    __device__ C<T> ld(int k) const {
        const int kk = k < Hx ? k : M0 - k;
        C<T> a = mk<T>(0, 0), b = mk<T>(0, 0);
        if (nr0) a = p[kk];
        if (nr1) b = p[Hx + kk];
        if (k >= Hx) {
            a.y = -a.y;
            b.y = -b.y;
        }
        return mk<T>(a.x - b.y, a.y + b.x);
    }
};
// xi output: element i of line p is (row 2p + i row 2p+1) at window cell
// w = (i - s0) mod M0 (and w + M0 when inside the window), times 1/(M0 M1 M2)
template <typename T> struct XiOut {
    T* __restrict__ p;               // row 2 line of this CTA
    int W0, s0, M0, nr0, nr1;
    T norm;
    __device__ void st(int i, C<T> v) const {
        int w = i - s0;
        if (w < 0) w += M0;
        for (; w < W0; w += M0) {
            if (nr0) p[w] = v.x * norm;
            if (nr1) p[W0 + w] = v.y * norm;
        }
    }
};

// xf: GMF rows -> half spectra along x, A[z][y][kx].  The CTA's 2 np GMF rows
// are one contiguous range of int64; when G0 is even and the range 16-byte
// aligned, one bulk asynchronous copy (TMA engine) stages it in shared memory
// while the twiddles load, completing on an mbarrier (bounded wait; a wait
// that runs out sets the status word's timeout bit and the CTA returns).
// Otherwise every thread loads its cells.  The cells are then converted and
// packed x-fastest.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, MinCtas<T>::value * (kFftThreads / NT)) k_xf(const GridDev* __restrict__ grids,
                                                    const Chunk* __restrict__ chunks,
                                                    const int64_t* const* __restrict__ gmf,
                                                    const C<T>* __restrict__ tw_arena,
                                                    C<T>* __restrict__ wsA, int F,
                                                    unsigned* __restrict__ status, int inject_wait) {
    extern __shared__ __align__(128) unsigned char smem_xf[];
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    const int M0 = g.M[0], G0 = g.G[0], Hx = g.Hx, np = g.lines[kPassXf], lg = ilog2(np), es = np + 1;
    const size_t stage = fft_xf_stage_bytes(np, G0);
    int64_t* rows = reinterpret_cast<int64_t*>(smem_xf);
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_xf + stage - 128);
    C<T>* cur = reinterpret_cast<C<T>*>(smem_xf + stage);
    C<T>* nxt = cur + M0 * es;
    C<T>* tw = nxt + M0 * es;
    // this CTA's rows: r_first + [0, nr), nr <= 2 np; 32-bit offsets from there
    const long long r_first = 2LL * ch.tile * np;
    const int nr = (int)min(2LL * np, (long long)g.G[1] * g.G[2] - r_first);
    const int64_t* __restrict__ in = gmf[ch.grid] + r_first * G0;
    const bool bulk = !(G0 & 1) && !(reinterpret_cast<size_t>(in) & 15);
    if (bulk) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            fence_proxy_async_smem();
            const unsigned bytes = (unsigned)nr * (unsigned)G0 * 8u;
            mbar_arrive_expect_tx(bar, bytes + (inject_wait ? 16u : 0u));
            bulk_g2s(rows, in, bytes, bar);
        }
    }
    load_twiddles<T, NT>(tw, tw_arena + g.fx.tw_off, M0);
    const int line = threadIdx.x & (np - 1);
    if (bulk) {
        __syncthreads();   // the barrier's initialisation is visible to every thread
        const bool ok = mbar_wait_bounded(bar, 0, kWaitPolls);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0 && status) atomicOr(status, kStTimeout);
            mbar_wait_bounded(bar, 0, kWaitPolls);   // the copy may still land: wait for it once more
            return;
        }
    }
    // cells packed x-fastest over threads: rows 2p, 2p+1 are complex line p
    {
        const T scale = pow2_neg<T>(F);
        const int64_t* src = bulk ? rows : in;
        int p = 0, x = threadIdx.x;
        while (x >= M0) { x -= M0; ++p; }
        const int dp = NT / M0, dx = NT % M0;
        for (; p < np; ) {
            const int q0 = 2 * p;
            T a = 0, b = 0;
            if (x < G0) {
                if (q0 < nr) a = fixed_to_real<T>(src[q0 * G0 + x], scale);
                if (q0 + 1 < nr) b = fixed_to_real<T>(src[(q0 + 1) * G0 + x], scale);
            }
            cur[x * es + p] = mk<T>(a, b);
            x += dx;
            p += dp;
            if (x >= M0) { x -= M0; ++p; }
        }
    }
    __syncthreads();
    const SmemIO<T> none{nullptr, 0, 0};
    stages_io<T, -1, NT, true, true>(g.fx, 0, g.fx.nst - 1, lg, tw, none, none, cur, nxt, es, line);
    // separate the two real rows: A_k = (Z_k + conj Z_{M-k}) / 2, B_k = (Z_k - conj Z_{M-k}) / 2i
    C<T>* out = wsA + (g.wsA + r_first * Hx);
    const C<T>* s = cur;
    {
        int p = 0, k = threadIdx.x;
        while (k >= Hx) { k -= Hx; ++p; }
        const int dp = NT / Hx, dk = NT % Hx;
        for (; p < np; ) {
            const int q0 = 2 * p;
            if (q0 < nr) {
                C<T> z = s[k * es + p];
                C<T> zm = s[(k == 0 ? 0 : M0 - k) * es + p];
                out[q0 * Hx + k] = mk<T>((T)0.5 * (z.x + zm.x), (T)0.5 * (z.y - zm.y));
                if (q0 + 1 < nr) out[(q0 + 1) * Hx + k] = mk<T>((T)0.5 * (z.y + zm.y), (T)0.5 * (zm.x - z.x));
            }
            k += dk;
            p += dp;
            if (k >= Hx) { k -= Hx; ++p; }
        }
    }
}

// xi: half spectra -> real rows of the window, C2R two rows per complex line
template <typename T, int NT>
__global__ void __launch_bounds__(NT, MinCtas<T>::value * (kFftThreads / NT)) k_xi(const GridDev* __restrict__ grids,
                                                    const Chunk* __restrict__ chunks,
                                                    const C<T>* __restrict__ tw_arena,
                                                    const C<T>* __restrict__ wsB,
                                                    void* const* __restrict__ phis, int comp) {
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    const int M0 = g.M[0], Hx = g.Hx, np = g.lines[kPassXi], W0 = g.W[0], lg = ilog2(np), es = np + 1;
    C<T>* cur = smem_c<T>();
    C<T>* nxt = cur + M0 * es;
    C<T>* tw = nxt + M0 * es;
    const long long r_first = 2LL * ch.tile * np;
    const int nr = (int)min(2LL * np, (long long)g.W[1] * g.W[2] - r_first);
    load_twiddles<T, NT>(tw, tw_arena + g.fx.tw_off, M0);
    const int line = threadIdx.x & (np - 1);
    XiIn<T> in;
    in.p = wsB + (g.wsB + (r_first + 2 * line) * Hx);
    in.Hx = Hx;
    in.M0 = M0;
    in.nr0 = 2 * line < nr;
    in.nr1 = 2 * line + 1 < nr;
    XiOut<T> out;
    // component comp of a spectral-gradient solve: the comp-th window of W cells
    out.p = reinterpret_cast<T*>(phis[ch.grid]) + (long long)comp * g.W[0] * g.W[1] * g.W[2] +
            (r_first + 2 * line) * W0;
    out.W0 = W0;
    out.s0 = g.s0[0];
    out.M0 = M0;
    out.nr0 = in.nr0;
    out.nr1 = in.nr1;
    out.norm = (T)g.inv_m3;
    __syncthreads();
    stages_io<T, 1, NT, false, false>(g.fx, 0, g.fx.nst - 1, lg, tw, in, out, cur, nxt, es, line);
}

}  // namespace
}  // namespace apm

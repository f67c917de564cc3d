// k_fft.cu -- batched 3-D FFT convolution of every grid of a level (Sec. 2.2,
// Eq. PoissonFourier): the zero-padded GMF of each grid is transformed on its
// M0 x M1 x M2 grid, multiplied by the Green's table and transformed back; only
// the window of cells [-2, N+2) of the result is written.
//
// Five passes, each one CTA per batch of lines, each line transformed entirely
// in shared memory by mixed-radix (2, 3, 4, 5, 7, 8) Stockham stages:
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
#include "apm_internal.cuh"

namespace apm {
namespace {

template <typename T> using C = typename Cplx<T>::type;

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

// In-register DFT of size R: X_q = sum_r v_r exp(DIR 2 pi i q r / R).
// `root` holds exp(DIR 2 pi i t / R), t < R (used by the odd radices).
template <typename T, int DIR, int R> struct Dft;

template <typename T, int DIR> struct Dft<T, DIR, 2> {
    __device__ static void run(C<T>* v, const C<T>*) {
        C<T> a = v[0], b = v[1];
        v[0] = add<T>(a, b);
        v[1] = sub<T>(a, b);
    }
};

template <typename T, int DIR> struct Dft<T, DIR, 4> {
    __device__ static void run(C<T>* v, const C<T>*) {
        C<T> t0 = add<T>(v[0], v[2]), t1 = sub<T>(v[0], v[2]);
        C<T> t2 = add<T>(v[1], v[3]), t3 = rot90<T, DIR>(sub<T>(v[1], v[3]));
        v[0] = add<T>(t0, t2);
        v[2] = sub<T>(t0, t2);
        v[1] = add<T>(t1, t3);
        v[3] = sub<T>(t1, t3);
    }
};

template <typename T, int DIR> struct Dft<T, DIR, 8> {
    __device__ static void run(C<T>* v, const C<T>*) {
        C<T> e[4] = {v[0], v[2], v[4], v[6]};
        C<T> o[4] = {v[1], v[3], v[5], v[7]};
        Dft<T, DIR, 4>::run(e, nullptr);
        Dft<T, DIR, 4>::run(o, nullptr);
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

// odd radices: direct sum with the roots of unity
template <typename T, int DIR, int R> struct Dft {
    __device__ static void run(C<T>* v, const C<T>* root) {
        C<T> out[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            C<T> acc = v[0];
#pragma unroll
            for (int r = 1; r < R; ++r) acc = add<T>(acc, mul<T>(v[r], root[(q * r) % R]));
            out[q] = acc;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = out[q];
    }
};

// One Stockham stage of radix R over `nl` lines of length L (element i of line
// l at [l*ls + i*es]), from src to dst in shared memory; Ns = product of the
// radices already applied.  Butterfly j reads elements j + r L/R, twiddles them
// by exp(DIR 2 pi i (j mod Ns) r / (Ns R)), and writes elements
// (j / Ns) Ns R + (j mod Ns) + r Ns: natural order after the last stage.
// lf: consecutive threads take consecutive lines (else consecutive butterflies).
template <typename T, int DIR, int R>
__device__ void stage(const C<T>* __restrict__ src, C<T>* __restrict__ dst, int L, int Ns, int nl,
                      int ls, int es, bool lf, const C<T>* __restrict__ tw) {
    const int nb = L / R;
    const int total = nb * nl;
    const int step = L / (Ns * R);
    C<T> root[R];
    if (R & 1) {
#pragma unroll
        for (int t = 0; t < R; ++t) root[t] = twid<T, DIR>(tw, t * nb);
    }
    for (int w = threadIdx.x; w < total; w += kFftThreads) {
        int line = lf ? w % nl : w / nb;
        int j = lf ? w / nl : w - (w / nb) * nb;
        const C<T>* s = src + line * ls;
        C<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[(j + r * nb) * es];
        int jm = j % Ns;
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = mul<T>(v[r], twid<T, DIR>(tw, jm * r * step));
        }
        Dft<T, DIR, R>::run(v, root);
        C<T>* d = dst + line * ls;
        int idx = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) d[(idx + r * Ns) * es] = v[r];
    }
    __syncthreads();
}

// Full transform of nl lines; the input is in `a`, `b` is scratch of the same
// size; returns the buffer holding the result.
template <typename T, int DIR>
__device__ C<T>* fft_lines(C<T>* a, C<T>* b, const FftPlan1D& pl, int nl, int ls, int es, bool lf,
                           const C<T>* tw_arena) {
    const C<T>* tw = tw_arena + pl.tw_off;
    const int L = pl.L;
    int Ns = 1;
    for (int st = 0; st < pl.nst; ++st) {
        int R = pl.radix[st];
        switch (R) {
            case 8: stage<T, DIR, 8>(a, b, L, Ns, nl, ls, es, lf, tw); break;
            case 4: stage<T, DIR, 4>(a, b, L, Ns, nl, ls, es, lf, tw); break;
            case 2: stage<T, DIR, 2>(a, b, L, Ns, nl, ls, es, lf, tw); break;
            case 3: stage<T, DIR, 3>(a, b, L, Ns, nl, ls, es, lf, tw); break;
            case 5: stage<T, DIR, 5>(a, b, L, Ns, nl, ls, es, lf, tw); break;
            default: stage<T, DIR, 7>(a, b, L, Ns, nl, ls, es, lf, tw); break;
        }
        C<T>* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// complex elements of one of the two shared-memory buffers of a CTA
template <typename T> struct Budget { static constexpr int value = kFftBudgetF32; };
template <> struct Budget<double> { static constexpr int value = kFftBudgetF64; };

template <typename T> __device__ __forceinline__ C<T>* smem_c() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<C<T>*>(smem_raw);
}

// ---- xf: GMF rows -> half spectra along x ----------------------------------
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_xf(const GridDev* __restrict__ grids,
                                                    const Chunk* __restrict__ chunks,
                                                    const int64_t* const* __restrict__ gmf,
                                                    const C<T>* __restrict__ tw, C<T>* __restrict__ wsA,
                                                    int F) {
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    C<T>* s = smem_c<T>();
    C<T>* s2 = s + Budget<T>::value;
    const int M0 = g.M[0], G0 = g.G[0], Hx = g.Hx, np = g.np_x;
    const long long nrows = (long long)g.G[1] * g.G[2];
    const long long r_first = 2LL * ch.tile * np;
    const int64_t* in = gmf[ch.grid];
    for (int e = threadIdx.x; e < np * M0; e += kFftThreads) {
        int p = e / M0, x = e - p * M0;
        long long r0 = r_first + 2 * p, r1 = r0 + 1;
        T a = 0, b = 0;
        if (x < G0) {
            if (r0 < nrows) a = (T)ldexp((double)in[r0 * G0 + x], -F);
            if (r1 < nrows) b = (T)ldexp((double)in[r1 * G0 + x], -F);
        }
        s[e] = mk<T>(a, b);
    }
    __syncthreads();
    s = fft_lines<T, -1>(s, s2, g.fx, np, M0, 1, false, tw);
    // separate the two real rows: A_k = (Z_k + conj Z_{M-k}) / 2, B_k = (Z_k - conj Z_{M-k}) / 2i
    C<T>* out = wsA + g.wsA;
    for (int e = threadIdx.x; e < np * Hx; e += kFftThreads) {
        int p = e / Hx, k = e - p * Hx;
        long long r0 = r_first + 2 * p, r1 = r0 + 1;
        if (r0 >= nrows) continue;
        C<T> z = s[p * M0 + k];
        C<T> zm = s[p * M0 + (k == 0 ? 0 : M0 - k)];
        out[r0 * Hx + k] = mk<T>((T)0.5 * (z.x + zm.x), (T)0.5 * (z.y - zm.y));
        if (r1 < nrows) out[r1 * Hx + k] = mk<T>((T)0.5 * (z.y + zm.y), (T)0.5 * (zm.x - z.x));
    }
}

// ---- column passes -----------------------------------------------------------
// AX = 1 (y) or 2 (z).  MODE 0: forward only; 1: forward, table, inverse; 2: inverse only.
//   yf (AX 1, MODE 0): in A[z][y][kx] (y < G1), out B[z][ky][kx]
//   z  (AX 2, MODE 1): in B[z][ky][kx] (z < G2), out A[zw][ky][kx]
//   yi (AX 1, MODE 2): in A[zw][ky][kx],         out B[zw][yw][kx]
template <typename T, int AX, int MODE>
__global__ void __launch_bounds__(kFftThreads) k_col(const GridDev* __restrict__ grids,
                                                     const Chunk* __restrict__ chunks,
                                                     const C<T>* __restrict__ tw,
                                                     const T* __restrict__ tab,
                                                     C<T>* __restrict__ wsA, C<T>* __restrict__ wsB) {
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    C<T>* s = smem_c<T>();
    C<T>* s2 = s + Budget<T>::value;
    const int Hx = g.Hx;
    const int tx = AX == 1 ? g.tx_y : g.tx_z;
    const int nkt = (Hx + tx - 1) / tx;
    const int kxt = ch.tile % nkt;
    const int other = ch.tile / nkt;    // z (yf), ky (z), zw (yi)
    const int kx0 = kxt * tx;
    const FftPlan1D& pl = AX == 1 ? g.fy : g.fz;
    const int L = pl.L;
    const int M1 = g.M[1];

    const C<T>* in;
    long long in_base, in_stride;
    int n_in;
    if (AX == 1 && MODE == 0) {
        in = wsA + g.wsA; n_in = g.G[1];
        in_base = (long long)other * g.G[1] * Hx; in_stride = Hx;
    } else if (AX == 2) {
        in = wsB + g.wsB; n_in = g.G[2];
        in_base = (long long)other * Hx; in_stride = (long long)M1 * Hx;
    } else {
        in = wsA + g.wsA; n_in = M1;
        in_base = (long long)other * M1 * Hx; in_stride = Hx;
    }
    for (int e = threadIdx.x; e < L * tx; e += kFftThreads) {
        int i = e / tx, line = e - i * tx;
        int kx = kx0 + line;
        C<T> v = mk<T>(0, 0);
        if (i < n_in && kx < Hx) v = in[in_base + i * in_stride + kx];
        s[e] = v;
    }
    __syncthreads();
    if (MODE == 2) {
        s = fft_lines<T, 1>(s, s2, pl, tx, 1, tx, true, tw);
    } else {
        s = fft_lines<T, -1>(s, s2, pl, tx, 1, tx, true, tw);
    }
    s2 = (s == smem_c<T>()) ? s + Budget<T>::value : smem_c<T>();
    if (MODE == 1) {
        // phi-hat = T(kappa) rho-hat; the table is even in every component
        const int ky = other;
        const int fy = ky <= M1 / 2 ? ky : M1 - ky;
        const T* tb = tab + g.tab_off + (long long)fy * Hx;
        const long long zst = (long long)g.Hy2 * Hx;
        for (int e = threadIdx.x; e < L * tx; e += kFftThreads) {
            int kz = e / tx, line = e - kz * tx;
            int kx = kx0 + line;
            if (kx >= Hx) continue;
            int fz = kz <= L / 2 ? kz : L - kz;
            T t = tb[fz * zst + kx];
            C<T> v = s[e];
            s[e] = mk<T>(v.x * t, v.y * t);
        }
        __syncthreads();
        s = fft_lines<T, 1>(s, s2, pl, tx, 1, tx, true, tw);
    }
    // store
    C<T>* out;
    long long out_base, out_stride;
    int n_out, s0;
    if (AX == 1 && MODE == 0) {
        out = wsB + g.wsB; n_out = M1; s0 = 0;
        out_base = (long long)other * M1 * Hx; out_stride = Hx;
    } else if (AX == 2) {
        out = wsA + g.wsA; n_out = g.W[2]; s0 = g.s0[2];
        out_base = (long long)other * Hx; out_stride = (long long)M1 * Hx;
    } else {
        out = wsB + g.wsB; n_out = g.W[1]; s0 = g.s0[1];
        out_base = (long long)other * g.W[1] * Hx; out_stride = Hx;
    }
    for (int e = threadIdx.x; e < n_out * tx; e += kFftThreads) {
        int o = e / tx, line = e - o * tx;
        int kx = kx0 + line;
        if (kx >= Hx) continue;
        int i = (s0 + o) % L;
        out[out_base + o * out_stride + kx] = s[i * tx + line];
    }
}

// ---- xi: half spectra -> real rows of the window -------------------------------
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_xi(const GridDev* __restrict__ grids,
                                                    const Chunk* __restrict__ chunks,
                                                    const C<T>* __restrict__ tw,
                                                    const C<T>* __restrict__ wsB,
                                                    void* const* __restrict__ phis) {
    const Chunk ch = chunks[blockIdx.x];
    const GridDev& g = grids[ch.grid];
    C<T>* s = smem_c<T>();
    C<T>* s2 = s + Budget<T>::value;
    const int M0 = g.M[0], Hx = g.Hx, np = g.np_x, W0 = g.W[0];
    const long long nrows = (long long)g.W[1] * g.W[2];
    const long long r_first = 2LL * ch.tile * np;
    const C<T>* in = wsB + g.wsB;
    // Z_k = A_k + i B_k with A, B extended by Hermitian symmetry
    for (int e = threadIdx.x; e < np * M0; e += kFftThreads) {
        int p = e / M0, k = e - p * M0;
        long long r0 = r_first + 2 * p, r1 = r0 + 1;
        int kk = k < Hx ? k : M0 - k;
        C<T> a = mk<T>(0, 0), b = mk<T>(0, 0);
        if (r0 < nrows) a = in[r0 * Hx + kk];
        if (r1 < nrows) b = in[r1 * Hx + kk];
        if (k >= Hx) { a.y = -a.y; b.y = -b.y; }
        s[e] = mk<T>(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    s = fft_lines<T, 1>(s, s2, g.fx, np, M0, 1, false, tw);
    const T norm = (T)(1.0 / ((double)g.M[0] * (double)g.M[1] * (double)g.M[2]));
    T* out = reinterpret_cast<T*>(phis[ch.grid]);
    for (int e = threadIdx.x; e < np * W0; e += kFftThreads) {
        int p = e / W0, xw = e - p * W0;
        long long r0 = r_first + 2 * p, r1 = r0 + 1;
        if (r0 >= nrows) continue;
        int x = (g.s0[0] + xw) % M0;
        C<T> z = s[p * M0 + x];
        out[r0 * W0 + xw] = z.x * norm;
        if (r1 < nrows) out[r1 * W0 + xw] = z.y * norm;
    }
}

}  // namespace

// Allows every pass kernel the full per-CTA shared-memory budget (above the
// 48 KB default for the FP64 instantiations).
cudaError_t fft_configure() {
    const int f32 = (int)(2 * kFftBudgetF32 * sizeof(float2));
    const int f64 = (int)(2 * kFftBudgetF64 * sizeof(double2));
    const void* fns32[] = {(const void*)k_xf<float>, (const void*)k_col<float, 1, 0>,
                           (const void*)k_col<float, 2, 1>, (const void*)k_col<float, 1, 2>,
                           (const void*)k_xi<float>};
    const void* fns64[] = {(const void*)k_xf<double>, (const void*)k_col<double, 1, 0>,
                           (const void*)k_col<double, 2, 1>, (const void*)k_col<double, 1, 2>,
                           (const void*)k_xi<double>};
    for (const void* f : fns32) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, f32);
        if (e != cudaSuccess) return e;
    }
    for (const void* f : fns64) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, f64);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_fft_xf(const FftArgs& a, const int64_t* const* gmf, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    k_xf<T><<<a.n_chunks, kFftThreads, a.smem, s>>>(a.g, a.chunks, gmf, (const C<T>*)a.tw,
                                                    (C<T>*)a.wsA, a.F);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_yf(const FftArgs& a, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    k_col<T, 1, 0><<<a.n_chunks, kFftThreads, a.smem, s>>>(a.g, a.chunks, (const C<T>*)a.tw,
                                                           (const T*)a.tab, (C<T>*)a.wsA, (C<T>*)a.wsB);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_z(const FftArgs& a, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    k_col<T, 2, 1><<<a.n_chunks, kFftThreads, a.smem, s>>>(a.g, a.chunks, (const C<T>*)a.tw,
                                                           (const T*)a.tab, (C<T>*)a.wsA, (C<T>*)a.wsB);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_yi(const FftArgs& a, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    k_col<T, 1, 2><<<a.n_chunks, kFftThreads, a.smem, s>>>(a.g, a.chunks, (const C<T>*)a.tw,
                                                           (const T*)a.tab, (C<T>*)a.wsA, (C<T>*)a.wsB);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_xi(const FftArgs& a, void* const* phis, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    k_xi<T><<<a.n_chunks, kFftThreads, a.smem, s>>>(a.g, a.chunks, (const C<T>*)a.tw,
                                                    (const C<T>*)a.wsB, phis);
    return cudaGetLastError();
}

#define APM_INST(T)                                                                       \
    template cudaError_t launch_fft_xf<T>(const FftArgs&, const int64_t* const*, cudaStream_t); \
    template cudaError_t launch_fft_yf<T>(const FftArgs&, cudaStream_t);                   \
    template cudaError_t launch_fft_z<T>(const FftArgs&, cudaStream_t);                    \
    template cudaError_t launch_fft_yi<T>(const FftArgs&, cudaStream_t);                   \
    template cudaError_t launch_fft_xi<T>(const FftArgs&, void* const*, cudaStream_t);
APM_INST(float)
APM_INST(double)
#undef APM_INST

}  // namespace apm

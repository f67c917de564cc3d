// k_fft_fast.cu -- launchers of the FP32 FFT passes with compile-time plans
// (fft_fast.cuh), one per length of APM_FAST_LENGTHS; compiled once per pass
// with -DAPM_FAST_MODE=0|1|2|3|4|5 (yf, z, yi, xf, xi, z of a spectral-gradient
// component) so the instantiations build in parallel.
#include "fft_fast.cuh"

#if !defined(APM_FAST_MODE)
#error "k_fft_fast.cu is compiled with -DAPM_FAST_MODE=0|1|2|3|4|5"
#endif

namespace apm {

namespace {
constexpr int kFastMode = APM_FAST_MODE;
constexpr bool kFastRow = kFastMode == 3 || kFastMode == 4;
constexpr int kFastAx = (kFastMode == 1 || kFastMode == 5) ? 2 : 1;
constexpr int kColMode = kFastMode == 5 ? 3 : kFastMode;   // k_col_fast's MODE
constexpr int kLines = kFastRow ? kFastNp : kFastTx;

template <int A, int B, int Cc>
constexpr auto kernel_of() {
    using P = FastPlan<A, B, Cc>;
    constexpr int NT = fast_threads(A, B, Cc, kLines);
    if constexpr (kFastMode == 3) return k_xf_fast<P, kFastNp, NT>;
    else if constexpr (kFastMode == 4) return k_xi_fast<P, kFastNp, NT>;
    else return k_col_fast<P, kFastAx, kColMode, kFastTx, NT>;
}

template <int L>
size_t smem_of() { return kFastRow ? fast_row_smem(L) : fast_col_smem(L); }

template <int L, int A, int B, int Cc>
cudaError_t launch_one(const FftArgs& a, const int64_t* const* gmf, void* const* phis, cudaStream_t s) {
    static_assert(FastPlan<A, B, Cc>::L == L, "plan length");
    constexpr int NT = fast_threads(A, B, Cc, kLines);
    const auto kern = kernel_of<A, B, Cc>();
    if constexpr (kFastMode == 3)
        kern<<<a.n_chunks, NT, smem_of<L>(), s>>>(a.g, a.chunks, gmf, (const float2*)a.tw, (float2*)a.wsA, a.F);
    else if constexpr (kFastMode == 4)
        kern<<<a.n_chunks, NT, smem_of<L>(), s>>>(a.g, a.chunks, (const float2*)a.tw, (const float2*)a.wsB, phis,
                                                  a.comp);
    else
        kern<<<a.n_chunks, NT, smem_of<L>(), s>>>(a.g, a.chunks, (const float2*)a.tw, (const float*)a.tab,
                                                  (float2*)a.wsA, (float2*)a.wsB, a.comp);
    return cudaGetLastError();
}

template <int L, int A, int B, int Cc>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(kernel_of<A, B, Cc>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_of<L>());
}

// the fused x + y forward (x-forward unit only), for the lengths whose plane
// fits the shared-memory limit
template <int L, int A, int B, int Cc>
constexpr bool xy_fits() { return (size_t)(L * (L / 2 + 1) + L) * 8 <= (size_t)kFftSmemLimit; }

template <int L, int A, int B, int Cc>
cudaError_t configure_xy() {
    if constexpr (kFastMode == 3 && xy_fits<L, A, B, Cc>())
        return cudaFuncSetAttribute(k_xy_fast<FastPlan<A, B, Cc>, kFastXyThreads>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fast_xy_smem(L));
    if constexpr (kFastMode == 4 && xy_fits<L, A, B, Cc>())
        return cudaFuncSetAttribute(k_yx_fast<FastPlan<A, B, Cc>, kFastXyThreads>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fast_xy_smem(L));
    return cudaSuccess;
}

cudaError_t configure_fast() {
    cudaError_t e = cudaSuccess;
#define APM_FAST_CASE(LL, A, B, C) \
    if (e == cudaSuccess) e = configure_one<LL, A, B, C>(); \
    if (e == cudaSuccess) e = configure_xy<LL, A, B, C>();
    APM_FAST_LENGTHS(APM_FAST_CASE)
#undef APM_FAST_CASE
    return e;
}

#if APM_FAST_MODE == 4
template <int L, int A, int B, int Cc>
cudaError_t launch_yx_one(const FftArgs& a, void* const* phis, cudaStream_t s) {
    if constexpr (xy_fits<L, A, B, Cc>()) {
        k_yx_fast<FastPlan<A, B, Cc>, kFastXyThreads><<<a.n_chunks, kFastXyThreads, fast_xy_smem(L), s>>>(
            a.g, a.chunks, (const float2*)a.tw, (const float2*)a.wsA, phis, a.comp);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}
#endif

#if APM_FAST_MODE == 3
template <int L, int A, int B, int Cc>
cudaError_t launch_xy_one(const FftArgs& a, const int64_t* const* gmf, cudaStream_t s) {
    if constexpr (xy_fits<L, A, B, Cc>()) {
        k_xy_fast<FastPlan<A, B, Cc>, kFastXyThreads><<<a.n_chunks, kFastXyThreads, fast_xy_smem(L), s>>>(
            a.g, a.chunks, gmf, (const float2*)a.tw, (float2*)a.wsB, a.F);
        return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}
#endif

cudaError_t launch_fast(int L, const FftArgs& a, const int64_t* const* gmf, void* const* phis, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    switch (L) {
#define APM_FAST_CASE(LL, A, B, C) \
    case LL: return launch_one<LL, A, B, C>(a, gmf, phis, s);
        APM_FAST_LENGTHS(APM_FAST_CASE)
#undef APM_FAST_CASE
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

#if APM_FAST_MODE == 0
cudaError_t fft_configure_fast_yf() { return configure_fast(); }
cudaError_t launch_fft_yf_fast(int L, const FftArgs& a, cudaStream_t s) {
    return launch_fast(L, a, nullptr, nullptr, s);
}
#elif APM_FAST_MODE == 1
cudaError_t fft_configure_fast_z() { return configure_fast(); }
cudaError_t launch_fft_z_fast(int L, const FftArgs& a, cudaStream_t s) { return launch_fast(L, a, nullptr, nullptr, s); }
#elif APM_FAST_MODE == 2
cudaError_t fft_configure_fast_yi() { return configure_fast(); }
cudaError_t launch_fft_yi_fast(int L, const FftArgs& a, cudaStream_t s) {
    return launch_fast(L, a, nullptr, nullptr, s);
}
#elif APM_FAST_MODE == 3
cudaError_t fft_configure_fast_xf() { return configure_fast(); }
cudaError_t launch_fft_xy_fast(int L, const FftArgs& a, const int64_t* const* gmf, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    switch (L) {
#define APM_FAST_CASE(LL, A, B, C) \
    case LL: return launch_xy_one<LL, A, B, C>(a, gmf, s);
        APM_FAST_LENGTHS(APM_FAST_CASE)
#undef APM_FAST_CASE
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_fft_xf_fast(int L, const FftArgs& a, const int64_t* const* gmf, cudaStream_t s) {
    return launch_fast(L, a, gmf, nullptr, s);
}
#elif APM_FAST_MODE == 5
cudaError_t fft_configure_fast_zg() { return configure_fast(); }
cudaError_t launch_fft_zgrad_fast(int L, const FftArgs& a, cudaStream_t s) {
    return launch_fast(L, a, nullptr, nullptr, s);
}
#else
cudaError_t fft_configure_fast_xi() { return configure_fast(); }
cudaError_t launch_fft_yx_fast(int L, const FftArgs& a, void* const* phis, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    switch (L) {
#define APM_FAST_CASE(LL, A, B, C) \
    case LL: return launch_yx_one<LL, A, B, C>(a, phis, s);
        APM_FAST_LENGTHS(APM_FAST_CASE)
#undef APM_FAST_CASE
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_fft_xi_fast(int L, const FftArgs& a, void* const* phis, cudaStream_t s) {
    return launch_fast(L, a, nullptr, phis, s);
}
#endif

}  // namespace apm

// k_fft_col.cu -- one column pass (yf, z, yi, or the z pass of a spectral-
// gradient component) of the batched FFT convolution in one precision:
// compiled once per (precision, pass) with -DAPM_COL_FP64=0|1
// -DAPM_COL_MODE=0|1|2|3 (yf, z, yi, z gradient), so the eight instantiations
// build in parallel.
#include "fft_core.cuh"

#if !defined(APM_COL_FP64) || !defined(APM_COL_MODE)
#error "k_fft_col.cu is compiled with -DAPM_COL_FP64=0|1 -DAPM_COL_MODE=0|1|2|3"
#endif

namespace apm {

#if APM_COL_FP64
using ColT = double;
#define APM_COL_NAME(base) base##_f64
#else
using ColT = float;
#define APM_COL_NAME(base) base##_f32
#endif

constexpr int kColAx = (APM_COL_MODE == 1 || APM_COL_MODE == 3) ? 2 : 1;
constexpr int kColMode = APM_COL_MODE;

namespace {
cudaError_t configure_col() {
    const void* fns[] = {(const void*)k_col<ColT, kColAx, kColMode, 128>,
                         (const void*)k_col<ColT, kColAx, kColMode, 256>};
    for (const void* f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemLimit);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_col(const FftArgs& a, cudaStream_t s) {
    using T = ColT;
    if (a.n_chunks <= 0) return cudaSuccess;
    if (a.threads == 128)
        k_col<T, kColAx, kColMode, 128><<<a.n_chunks, 128, a.smem, s>>>(
            a.g, a.chunks, (const C<T>*)a.tw, (const T*)a.tab, (C<T>*)a.wsA, (C<T>*)a.wsB, a.comp);
    else
        k_col<T, kColAx, kColMode, 256><<<a.n_chunks, 256, a.smem, s>>>(
            a.g, a.chunks, (const C<T>*)a.tw, (const T*)a.tab, (C<T>*)a.wsA, (C<T>*)a.wsB, a.comp);
    return cudaGetLastError();
}
}  // namespace

#if APM_COL_MODE == 0
cudaError_t APM_COL_NAME(fft_configure_yf)() { return configure_col(); }
template <> cudaError_t launch_fft_yf<ColT>(const FftArgs& a, cudaStream_t s) { return launch_col(a, s); }
#elif APM_COL_MODE == 1
cudaError_t APM_COL_NAME(fft_configure_z)() { return configure_col(); }
template <> cudaError_t launch_fft_z<ColT>(const FftArgs& a, cudaStream_t s) { return launch_col(a, s); }
#elif APM_COL_MODE == 2
cudaError_t APM_COL_NAME(fft_configure_yi)() { return configure_col(); }
template <> cudaError_t launch_fft_yi<ColT>(const FftArgs& a, cudaStream_t s) { return launch_col(a, s); }
#else
cudaError_t APM_COL_NAME(fft_configure_zg)() { return configure_col(); }
template <> cudaError_t launch_fft_zgrad<ColT>(const FftArgs& a, cudaStream_t s) { return launch_col(a, s); }
#endif

}  // namespace apm

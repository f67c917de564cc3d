// k_fft_x.cu -- the x passes (xf, xi) of the batched FFT convolution and the
// shared-memory set-up of every pass kernel.
#include "fft_core.cuh"

namespace apm {

// the column passes' set-up (k_fft_col.cu, one per precision and pass)
cudaError_t fft_configure_yf_f32();
cudaError_t fft_configure_z_f32();
cudaError_t fft_configure_yi_f32();
cudaError_t fft_configure_yf_f64();
cudaError_t fft_configure_z_f64();
cudaError_t fft_configure_yi_f64();
cudaError_t fft_configure_zg_f32();
cudaError_t fft_configure_zg_f64();
// the FP32 passes with compile-time plans (k_fft_fast.cu)
cudaError_t fft_configure_fast_yf();
cudaError_t fft_configure_fast_z();
cudaError_t fft_configure_fast_yi();
cudaError_t fft_configure_fast_xf();
cudaError_t fft_configure_fast_xi();
cudaError_t fft_configure_fast_zg();

// Allows every pass kernel up to kFftSmemLimit of dynamic shared memory
// (above the 48 KB default).
cudaError_t fft_configure() {
    const void* fns[] = {(const void*)k_xf<float, 128>, (const void*)k_xf<float, 256>,
                         (const void*)k_xi<float, 128>, (const void*)k_xi<float, 256>,
                         (const void*)k_xf<double, 128>, (const void*)k_xf<double, 256>,
                         (const void*)k_xi<double, 128>, (const void*)k_xi<double, 256>};
    for (const void* f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemLimit);
        if (e != cudaSuccess) return e;
    }
    cudaError_t (*cols[])() = {fft_configure_yf_f32, fft_configure_z_f32, fft_configure_yi_f32,
                               fft_configure_zg_f32, fft_configure_yf_f64, fft_configure_z_f64,
                               fft_configure_yi_f64, fft_configure_zg_f64, fft_configure_fast_yf,
                               fft_configure_fast_z, fft_configure_fast_yi, fft_configure_fast_xf,
                               fft_configure_fast_xi, fft_configure_fast_zg};
    for (auto f : cols) {
        cudaError_t e = f();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The CTA size is a template parameter of the pass kernels (128 or 256 threads).
template <typename T>
cudaError_t launch_fft_xf(const FftArgs& a, const int64_t* const* gmf, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    if (a.threads == 128)
        k_xf<T, 128><<<a.n_chunks, 128, a.smem, s>>>(a.g, a.chunks, gmf, (const C<T>*)a.tw, (C<T>*)a.wsA, a.F,
                                                      a.status, a.inject_wait);
    else
        k_xf<T, 256><<<a.n_chunks, 256, a.smem, s>>>(a.g, a.chunks, gmf, (const C<T>*)a.tw, (C<T>*)a.wsA, a.F,
                                                      a.status, a.inject_wait);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft_xi(const FftArgs& a, void* const* phis, cudaStream_t s) {
    if (a.n_chunks <= 0) return cudaSuccess;
    if (a.threads == 128)
        k_xi<T, 128><<<a.n_chunks, 128, a.smem, s>>>(a.g, a.chunks, (const C<T>*)a.tw, (const C<T>*)a.wsB, phis, a.comp);
    else
        k_xi<T, 256><<<a.n_chunks, 256, a.smem, s>>>(a.g, a.chunks, (const C<T>*)a.tw, (const C<T>*)a.wsB, phis, a.comp);
    return cudaGetLastError();
}

template cudaError_t launch_fft_xf<float>(const FftArgs&, const int64_t* const*, cudaStream_t);
template cudaError_t launch_fft_xf<double>(const FftArgs&, const int64_t* const*, cudaStream_t);
template cudaError_t launch_fft_xi<float>(const FftArgs&, void* const*, cudaStream_t);
template cudaError_t launch_fft_xi<double>(const FftArgs&, void* const*, cudaStream_t);

}  // namespace apm

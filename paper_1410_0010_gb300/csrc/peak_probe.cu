// peak_probe.cu -- measured compute denominators of this GPU for the kernels
// that are not bound by HBM bandwidth: FP32 and FP64 fused multiply-add rates,
// the INT32 multiply-add rate, the warp-instruction issue rate, and the rate
// of 64-bit integer reductions to global memory (the deposit's red.add.u64).
// A standalone program (not part of libapm): prints one JSON object.
//
// Every kernel runs a fixed number of independent operations per thread (no
// waits, no data-dependent loop bounds) on a grid of 8 CTAs per SM, timed with
// CUDA events after a warm launch; the best of five launches is kept.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

namespace {

constexpr int kThreads = 256;
constexpr int kIters = 4096;   // loop trips per thread (FP32, INT32)
constexpr int kIters64 = 64;   // ... and FP64 (its rate is a small fraction of FP32's)
constexpr int kChains = 8;     // independent accumulators per thread

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma(T* out, T a, T b, int iters) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = acc[c] * a + b;   // one FMA each
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (T)-1.2345) out[0] = s;   // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(kThreads) k_imad(unsigned* out, unsigned a, unsigned b, int iters) {
    unsigned acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = acc[c] * a + b;   // one IMAD each
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= acc[c];
    if (s == 0x9e3779b9u) out[0] = s;
}

// 64-bit reductions spread over the first n words of a buffer: thread t adds
// to word (t * 7919 + it * 65599) mod n
__global__ void __launch_bounds__(kThreads) k_red(unsigned long long* buf, unsigned n, int iters) {
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int it = 0; it < iters; ++it) {
        const unsigned idx = (t * 7919u + (unsigned)it * 65599u) % n;
        asm volatile("red.global.add.u64 [%0], %1;" ::"l"(buf + idx), "l"(1ULL));
    }
}

#define CHECK(x)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (x);                                                     \
        if (e_ != cudaSuccess) {                                                  \
            std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));         \
            std::exit(1);                                                         \
        }                                                                         \
    } while (0)

template <typename F>
float best_ms(F launch) {
    cudaEvent_t e0, e1;
    CHECK(cudaEventCreate(&e0));
    CHECK(cudaEventCreate(&e1));
    launch();   // warm
    CHECK(cudaDeviceSynchronize());
    float best = 1e30f;
    for (int k = 0; k < 5; ++k) {
        CHECK(cudaEventRecord(e0));
        launch();
        CHECK(cudaEventRecord(e1));
        CHECK(cudaEventSynchronize(e1));
        float ms = 0;
        CHECK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) best = ms;
    }
    CHECK(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

int main() {
    cudaDeviceProp prop;
    CHECK(cudaGetDeviceProperties(&prop, 0));
    const int sms = prop.multiProcessorCount;
    const int blocks = sms * 8;
    const double threads = (double)blocks * kThreads;
    const double ops = threads * kIters * kChains;   // FMAs / IMADs per launch
    const double ops64 = threads * kIters64 * kChains;
    float* f32 = nullptr;
    double* f64 = nullptr;
    unsigned* u32 = nullptr;
    CHECK(cudaMalloc(&f32, sizeof(float)));
    CHECK(cudaMalloc(&f64, sizeof(double)));
    CHECK(cudaMalloc(&u32, sizeof(unsigned)));
    const float ms32 = best_ms([&] { k_fma<float><<<blocks, kThreads>>>(f32, 0.999f, 1e-3f, kIters); });
    const float ms64 = best_ms([&] { k_fma<double><<<blocks, kThreads>>>(f64, 0.999, 1e-3, kIters64); });
    const float msi = best_ms([&] { k_imad<<<blocks, kThreads>>>(u32, 2654435761u, 12345u, kIters); });
    // reductions: 64 Mi words (512 MB), 64 per thread
    const unsigned nwords = 64u << 20;
    const int red_iters = 64;
    unsigned long long* buf = nullptr;
    CHECK(cudaMalloc(&buf, (size_t)nwords * sizeof(unsigned long long)));
    CHECK(cudaMemset(buf, 0, (size_t)nwords * sizeof(unsigned long long)));
    const float msr = best_ms([&] { k_red<<<blocks, kThreads>>>(buf, nwords, red_iters); });
    // the same reductions into 4 Mi words (32 MB): the lines stay in L2, as the
    // deposit's mostly do (neighbouring particles share cloud cells)
    const unsigned nwords_l2 = 4u << 20;
    const float msr_l2 = best_ms([&] { k_red<<<blocks, kThreads>>>(buf, nwords_l2, red_iters); });
    int clock_khz = 0;
    CHECK(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, 0));
    // the FMA loops issue one warp instruction per 32 FMAs (plus loop control,
    // amortised over kChains): the FP32 figure bounds the issue rate from below
    const double fp32 = 2.0 * ops / (ms32 * 1e-3) / 1e12;
    const double fp64 = 2.0 * ops64 / (ms64 * 1e-3) / 1e12;
    const double int32 = ops / (msi * 1e-3) / 1e12;
    const double warp_issue = ops / 32.0 / (ms32 * 1e-3) / 1e9;
    const double red = threads * red_iters / (msr * 1e-3) / 1e9;
    const double red_l2 = threads * red_iters / (msr_l2 * 1e-3) / 1e9;
    std::printf("{\"gpu\": \"%s\", \"sms\": %d, \"sm_clock_max_mhz\": %.0f, "
                "\"fp32_fma_tflops\": %.2f, \"fp64_fma_tflops\": %.3f, \"int32_imad_tops\": %.2f, "
                "\"fp32_fma_warp_inst_per_s_e9\": %.1f, \"red_global_u64_per_s_e9\": %.1f, "
                "\"red_global_u64_l2_resident_per_s_e9\": %.1f, "
                "\"ms\": {\"fp32\": %.4f, \"fp64\": %.4f, \"int32\": %.4f, \"red\": %.4f, \"red_l2\": %.4f}}\n",
                prop.name, sms, clock_khz / 1e3, fp32, fp64, int32, warp_issue, red, red_l2, ms32, ms64, msi, msr,
                msr_l2);
    cudaFree(f32);
    cudaFree(f64);
    cudaFree(u32);
    cudaFree(buf);
    return 0;
}

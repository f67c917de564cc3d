// k_evolve.cu -- one timestep of the particles given accelerations evaluated at
// the half-step drifted positions x + v dt/2 (the drift of Sec. 2 that the
// deposit and interpolation apply): v' = v + a dt, x' = x + ((v + v')/2) dt,
// the drift-kick-drift leapfrog used to evolve the tests of Sec. 3.1 and 3.5
// without subcycling.  Every FP64 operation is explicitly rounded in this
// order, so the update is bit-identical to a plain IEEE evaluation.
#include "apm_internal.cuh"

namespace apm {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_kick_drift(long long n, double* __restrict__ x, double* __restrict__ y,
                                                    double* __restrict__ z, double* __restrict__ vx,
                                                    double* __restrict__ vy, double* __restrict__ vz,
                                                    const T* __restrict__ acc, double dt) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    double* pos[3] = {x, y, z};
    double* vel[3] = {vx, vy, vz};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const double v = vel[j][p];
        const double a = (double)acc[j * n + p];
        const double vn = __dadd_rn(v, __dmul_rn(a, dt));
        const double vm = __dmul_rn(__dadd_rn(v, vn), 0.5);
        pos[j][p] = __dadd_rn(pos[j][p], __dmul_rn(vm, dt));
        vel[j][p] = vn;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_kick_drift(long long n, double* x, double* y, double* z, double* vx, double* vy, double* vz,
                              const void* acc, double dt, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_kick_drift<T><<<blocks, 256, 0, s>>>(n, x, y, z, vx, vy, vz, reinterpret_cast<const T*>(acc), dt);
    return cudaGetLastError();
}

template cudaError_t launch_kick_drift<float>(long long, double*, double*, double*, double*, double*, double*,
                                              const void*, double, cudaStream_t);
template cudaError_t launch_kick_drift<double>(long long, double*, double*, double*, double*, double*, double*,
                                               const void*, double, cudaStream_t);

}  // namespace apm

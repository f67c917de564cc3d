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
    // all nine loads first (the arrays are distinct), then the updates
    const double v[3] = {vx[p], vy[p], vz[p]};
    const double q[3] = {x[p], y[p], z[p]};
    const double a[3] = {(double)acc[p], (double)acc[n + p], (double)acc[2 * n + p]};
    double vn[3], qn[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        vn[j] = __dadd_rn(v[j], __dmul_rn(a[j], dt));
        const double vm = __dmul_rn(__dadd_rn(v[j], vn[j]), 0.5);
        qn[j] = __dadd_rn(q[j], __dmul_rn(vm, dt));
    }
    x[p] = qn[0];
    y[p] = qn[1];
    z[p] = qn[2];
    vx[p] = vn[0];
    vy[p] = vn[1];
    vz[p] = vn[2];
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

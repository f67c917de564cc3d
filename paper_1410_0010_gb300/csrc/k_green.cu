// k_green.cu -- FFT twiddles and the APM Green's-function tables (FP64).
//
// Table entries are in DFT units: phi = IDFT( T * DFT(cell mass) ) / (M0 M1 M2),
// T = G-hat(k) / delta^3, stored on the octant kappa_j in [0, M_j/2] (x fastest);
// G-hat is even in every component, so the octant holds the whole table.
#include "apm_internal.cuh"

namespace apm {
namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Smoothing function of Sec. 2.2 Eq. S2k, S-hat(eta) = 12/eta^4 (2 - 2 cos eta -
// eta sin eta).  Below eta = 1 the closed form cancels; there its Taylor series
// 12 sum_{m>=2} (-1)^m (2m-2)/(2m)! eta^(2m-4) is summed (m = 2..13).
__device__ double shat(double eta) {
    if (eta < 1.0) {
        double e2 = eta * eta;
        double fact = 24.0, pw = 1.0, sum = 0.0;
        for (int m = 2; m <= 13; ++m) {
            if (m > 2) {
                fact *= (double)(2 * m - 1) * (double)(2 * m);
                pw *= e2;
            }
            double term = (double)(2 * m - 2) / fact * pw;
            sum += (m & 1) ? -term : term;
        }
        return 12.0 * sum;
    }
    double e2 = eta * eta;
    return 12.0 / (e2 * e2) * (2.0 - 2.0 * cos(eta) - eta * sin(eta));
}

// sinc(pi f) = sin(pi f) / (pi f)
__device__ double sinc_pi(double f) { return f == 0.0 ? 1.0 : sinpi(f) / (kPi * f); }

// Gradient operator at the centred mode kc = f M of an M grid (apm_gradient):
// two-point sin(k delta)/delta, four-point sin(k delta)(4 - cos(k delta))/(3 delta)
// (the symbol of the (8, -1)/12 stencil), spectral k with 0 on the Nyquist
// mode of an even M.  The factor -i common to all is left out.
__device__ double grad_symbol(int grad, int kc, int M, double delta) {
    const double f = (double)kc / (double)M;
    if (grad == APM_GRAD_FD2) return sinpi(2.0 * f) / delta;
    if (grad == APM_GRAD_FD4) return sinpi(2.0 * f) * (4.0 - cospi(2.0 * f)) / (3.0 * delta);
    return 2 * kc == M ? 0.0 : 2.0 * kPi * f / delta;
}

// Optimal influence function (Sec. 2.2 Eq. influence) at integer mode kap of an
// M grid with cell delta, TSC assignment (Eq. assignment read as U^2 =
// prod sinc^6, alias sum Eq. assignment2), gradient D = grad_symbol, Brillouin
// zones n in [-1,1]^3 (Eq. brillouin), and reference force S(a_lev)^2/k^2
// minus, on refined levels, S(a_par)^2/k^2 (Eq. reference).  Continuum units
// (potential per unit density).
__device__ double green_opt(const int kap[3], const int M[3], double delta, double a_lev,
                            double a_par, bool use_parent, int grad) {
    double f[3], k[3], D[3];
    double alias = 1.0, D2 = 0.0;
    for (int j = 0; j < 3; ++j) {
        int kc = kap[j] > M[j] / 2 ? kap[j] - M[j] : kap[j];
        f[j] = (double)kc / (double)M[j];
        k[j] = 2.0 * kPi * f[j] / delta;
        D[j] = grad_symbol(grad, kc, M[j], delta);
        double s = sinpi(f[j]);
        double s2 = s * s;
        alias *= 1.0 - s2 + (2.0 / 15.0) * s2 * s2;
        D2 += D[j] * D[j];
    }
    double num = 0.0;
    for (int n2 = -1; n2 <= 1; ++n2)
        for (int n1 = -1; n1 <= 1; ++n1)
            for (int n0 = -1; n0 <= 1; ++n0) {
                const int n[3] = {n0, n1, n2};
                double U2 = 1.0, Dq = 0.0, qq = 0.0;
                for (int j = 0; j < 3; ++j) {
                    double qj = k[j] + 2.0 * kPi * (double)n[j] / delta;
                    double sc = sinc_pi(f[j] + (double)n[j]);
                    double sc2 = sc * sc;
                    U2 *= sc2 * sc2 * sc2;
                    Dq += D[j] * qj;
                    qq += qj * qj;
                }
                double q = sqrt(qq);
                double sl = shat(q * a_lev * 0.5);
                double F = sl * sl / qq;
                if (use_parent) {
                    double sp = shat(q * a_par * 0.5);
                    F -= sp * sp / qq;
                }
                num += U2 * Dq * F;
            }
    return -4.0 * kPi * num / (D2 * alias * alias);
}

// modes where every operator's gradient vanishes identically (reading R5)
__device__ bool fd_degenerate(const int kap[3], const int M[3]) {
    for (int j = 0; j < 3; ++j)
        if (!(kap[j] == 0 || 2 * kap[j] == M[j])) return false;
    return true;
}

struct Oct {
    int M[3], H[3];
};

__device__ void oct_index(long long i, const Oct& o, int kap[3]) {
    kap[0] = (int)(i % o.H[0]);
    long long r = i / o.H[0];
    kap[1] = (int)(r % o.H[1]);
    kap[2] = (int)(r / o.H[1]);
}

// kind 0 (refined level) and kind 1 (periodic root) tables
__global__ void k_green_opt(int kind, Oct o, double delta, double a_lev, double a_par, int grad,
                            double* __restrict__ out) {
    long long total = (long long)o.H[0] * o.H[1] * o.H[2];
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    int kap[3];
    oct_index(i, o, kap);
    double vol = (delta * delta) * delta;
    bool zero = kap[0] == 0 && kap[1] == 0 && kap[2] == 0;
    double v = 0.0;
    if (kind == 0) {
        if (zero)
            v = -4.0 * kPi * (a_par * a_par - a_lev * a_lev) / 30.0 / vol;  // k -> 0 limit
        else if (!fd_degenerate(kap, o.M))
            v = green_opt(kap, o.M, delta, a_lev, a_par, true, grad) / vol;
    } else {
        if (!zero && !fd_degenerate(kap, o.M)) v = green_opt(kap, o.M, delta, a_lev, 0.0, false, grad) / vol;
    }
    out[i] = v;
}

// Pair potential of two unit-mass S spheres of diameter a (G = 1) at r = xi a,
// times a: the real-space kernel whose transform is -4 pi S-hat^2/k^2.
__device__ double pair_potential(double xi) {
    if (xi <= 0.5) {
        double x2 = xi * xi, x4 = x2 * x2;
        return -104.0 / 35.0 + 32.0 / 5.0 * x2 - 64.0 / 5.0 * x4 + 32.0 / 5.0 * x4 * xi +
               256.0 / 35.0 * x4 * x2 - 192.0 / 35.0 * x4 * x2 * xi;
    }
    if (xi <= 1.0) {
        double x2 = xi * xi, x3 = x2 * xi, x4 = x2 * x2;
        return -3.0 / (35.0 * xi) - 64.0 / 35.0 - 32.0 / 5.0 * xi + 128.0 / 5.0 * x2 - 32.0 * x3 +
               64.0 / 5.0 * x4 + 32.0 / 5.0 * x4 * xi - 256.0 / 35.0 * x4 * x2 +
               64.0 / 35.0 * x4 * x3;
    }
    return -1.0 / xi;
}

// Isolated root: kernel at the minimum-image offsets d in [0, M/2]^3 of the
// doubled grid (the rest follows by evenness).
__global__ void k_pair_octant(Oct o, double delta, double a, double* __restrict__ out) {
    long long total = (long long)o.H[0] * o.H[1] * o.H[2];
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    int d[3];
    oct_index(i, o, d);
    double r2 = 0.0;
    for (int j = 0; j < 3; ++j) {
        double rj = (double)d[j] * delta;
        r2 += rj * rj;
    }
    out[i] = pair_potential(sqrt(r2) / a) / a;
}

// DFT along `axis` of a real field that is even along that axis, stored on the
// octant: out(kappa) = sum_{d=0}^{M-1} g(d) cos(2 pi kappa d / M), folding the
// offsets d and M - d onto the stored d <= M/2.
__global__ void k_even_dft_axis(Oct o, int axis, const double* __restrict__ in,
                                double* __restrict__ out) {
    long long total = (long long)o.H[0] * o.H[1] * o.H[2];
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    int kap[3];
    oct_index(i, o, kap);
    const int M = o.M[axis];
    const int H = o.H[axis];
    long long stride = axis == 0 ? 1 : (axis == 1 ? o.H[0] : (long long)o.H[0] * o.H[1]);
    long long base = i - (long long)kap[axis] * stride;
    const int kk = kap[axis];
    double s = 0.0;
    for (int d = 0; d < H; ++d) {
        double w = (d == 0 || 2 * d == M) ? 1.0 : 2.0;
        int t = (int)(((long long)kk * d) % M);
        s += w * in[base + (long long)d * stride] * cospi(2.0 * (double)t / (double)M);
    }
    out[i] = s;
}

// adds the k-space optimal correction G_opt - (-4 pi S^2/k^2) on non-degenerate
// modes kappa != 0 (isolated root, optional)
__global__ void k_iso_correction(Oct o, double delta, double a, int grad, double* __restrict__ io) {
    long long total = (long long)o.H[0] * o.H[1] * o.H[2];
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    int kap[3];
    oct_index(i, o, kap);
    if ((kap[0] == 0 && kap[1] == 0 && kap[2] == 0) || fd_degenerate(kap, o.M)) return;
    double kk = 0.0;
    for (int j = 0; j < 3; ++j) {
        double kj = 2.0 * kPi * (double)kap[j] / ((double)o.M[j] * delta);
        kk += kj * kj;
    }
    double s = shat(sqrt(kk) * a * 0.5);
    double cont = -4.0 * kPi * s * s / kk;
    double vol = (delta * delta) * delta;
    io[i] += (green_opt(kap, o.M, delta, a, 0.0, false, grad) - cont) / vol;
}

__global__ void k_twiddles(double2* __restrict__ tw64, float2* __restrict__ tw32, int L) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)L, &s, &c);
    tw64[t] = make_double2(c, -s);
    tw32[t] = make_float2((float)c, (float)-s);
}

__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_twiddles(double2* tw64, float2* tw32, int L, cudaStream_t s) {
    k_twiddles<<<blocks_for(L, 256), 256, 0, s>>>(tw64, tw32, L);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* in, float* out, long long n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_to_f32<<<blocks_for(n, 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_green_table(int kind, const int M[3], double delta, double a_lev, double a_par,
                               int correction, int grad, double* out, double* scratch, cudaStream_t s) {
    Oct o;
    for (int j = 0; j < 3; ++j) {
        o.M[j] = M[j];
        o.H[j] = M[j] / 2 + 1;
    }
    long long total = (long long)o.H[0] * o.H[1] * o.H[2];
    const int T = 128;
    if (kind == 0 || kind == 1) {
        k_green_opt<<<blocks_for(total, T), T, 0, s>>>(kind, o, delta, a_lev, a_par, grad, out);
        return cudaGetLastError();
    }
    // isolated root: transform of the real-space kernel, axis by axis
    k_pair_octant<<<blocks_for(total, T), T, 0, s>>>(o, delta, a_lev, out);
    k_even_dft_axis<<<blocks_for(total, T), T, 0, s>>>(o, 0, out, scratch);
    k_even_dft_axis<<<blocks_for(total, T), T, 0, s>>>(o, 1, scratch, out);
    k_even_dft_axis<<<blocks_for(total, T), T, 0, s>>>(o, 2, out, scratch);
    cudaError_t e = cudaMemcpyAsync(out, scratch, total * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (correction) k_iso_correction<<<blocks_for(total, T), T, 0, s>>>(o, delta, a_lev, grad, out);
    return cudaGetLastError();
}

}  // namespace apm

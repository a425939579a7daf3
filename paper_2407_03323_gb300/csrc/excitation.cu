// Tested incident field (Eq. E) on the GPU:
//   E^b_{m,n} = chi_m p_b (1/V) int_{V_m} g(n dt - t0 - r . k_hat) dV,
//   g(tau) = sin(2 pi f_c tau) exp(-tau^2 / (2 sigma_t^2)),
// voxel m occupying [u, u+1] x [v, v+1] x [w, w+1] (h = c dt = 1).  The voxel average
// is a 6-point-per-axis tensor Gauss-Legendre rule; the pulse varies on a scale of
// many voxels so the rule is exact to rounding.
#include "mot_internal.cuh"

namespace {

constexpr int NQ = 6;
__constant__ double c_qx[NQ], c_qw[NQ];

__global__ void k_plane_wave(long long M, int U, int V, const double* __restrict__ chi, double kx,
                             double ky, double kz, double px, double py, double pz, double fc,
                             double st, double t0, int n_first, int n_steps,
                             double* __restrict__ E) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * n_steps) return;
    const long long m = i % M;
    const int step = (int)(i / M);
    const double ch = chi[m];
    double* o = E + i * 3;
    if (ch == 0.0) { o[0] = o[1] = o[2] = 0.0; return; }
    const int u = (int)(m % U), v = (int)((m / U) % V), w = (int)(m / ((long long)U * V));
    const double tc = (double)(n_first + step) - t0 -
                      ((u + 0.5) * kx + (v + 0.5) * ky + (w + 0.5) * kz);
    const double inv2s2 = 1.0 / (2.0 * st * st);
    double acc = 0.0;
    for (int a = 0; a < NQ; ++a)
        for (int b = 0; b < NQ; ++b)
            for (int c = 0; c < NQ; ++c) {
                const double tau = tc - (c_qx[a] * kx + c_qx[b] * ky + c_qx[c] * kz);
                acc += c_qw[a] * c_qw[b] * c_qw[c] * sinpi(2.0 * fc * tau) * exp(-tau * tau * inv2s2);
            }
    const double g = ch * acc;
    o[0] = g * px;
    o[1] = g * py;
    o[2] = g * pz;
}

}  // namespace

namespace mot {

void plane_wave(mot_ctx* c, const double k[3], const double p[3], double fc, double st, double t0,
                int n_first, int n_steps, double* Edev, cudaStream_t s) {
    // Gauss-Legendre nodes on [-1/2, 1/2] (weights sum to 1)
    double x[NQ], w[NQ];
    {
        const double pi = 3.14159265358979323846;
        for (int i = 0; i < NQ; ++i) {
            double z = std::cos(pi * (i + 0.75) / (NQ + 0.5)), dp = 0.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int kk = 2; kk <= NQ; ++kk) {
                    const double p2 = ((2.0 * kk - 1.0) * z * p1 - (kk - 1.0) * p0) / kk;
                    p0 = p1;
                    p1 = p2;
                }
                dp = NQ * (z * p1 - p0) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-17) break;
            }
            x[i] = 0.5 * z;
            w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
        }
    }
    MOT_CUDA_TRY(cudaMemcpyToSymbol(c_qx, x, sizeof x));
    MOT_CUDA_TRY(cudaMemcpyToSymbol(c_qw, w, sizeof w));
    const long long tot = c->M * n_steps;
    k_plane_wave<<<(int)((tot + 255) / 256), 256, 0, s>>>(c->M, c->U, c->V, c->chi, k[0], k[1], k[2],
                                                          p[0], p[1], p[2], fc, st, t0, n_first,
                                                          n_steps, Edev);
    MOT_LAUNCH_CHECK();
}

}  // namespace mot

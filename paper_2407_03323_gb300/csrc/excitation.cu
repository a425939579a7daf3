// Tested incident field (Eq. E) on the GPU:
//   E^b_{m,n} = chi_m p_b (1/V) int_{V_m} g(n dt - t0 - r . k_hat) dV,
//   g(tau) = sin(2 pi f_c tau) exp(-tau^2 / (2 sigma_t^2)),
// voxel m occupying [u, u+1] x [v, v+1] x [w, w+1] (h = c dt = 1).  The voxel average
// is a 6-point-per-axis tensor Gauss-Legendre rule; the pulse varies on a scale of
// many voxels so the rule is exact to rounding.
//
// The average A(tau) = int_{[-1/2,1/2]^3} g(tau - q . k_hat) dq is one function of
// tau = n dt - t0 - r_c . k_hat (r_c the voxel centre) for every voxel, so it is
// tabulated once per call on the nodes j h (j integer) covering every needed tau
// (the tensor rule at each node) and each voxel and step interpolates it: barycentric
// Lagrange form through the 10 nearest nodes (degree 9, equispaced weights
// (-1)^j C(9, j)).  With f_eff = f_c + 6 / (2 pi sigma_t) bounding the pulse's
// spectrum, the interpolation error is at most (2 pi f_eff h)^10 * 870 / 10! of max|g|;
// h = min(0.5, 0.057 / (2 pi f_eff)) keeps it below 1e-16, under the rule's rounding.
#include "mot_internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

namespace {

constexpr int NQ = 6;
constexpr int kMaxSetupDevices = 64;
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

// A((j0 + j) h), j < J, by the tensor rule (nodes on the fixed lattice h Z, so a value
// does not depend on which call tabulates it)
__global__ void k_pw_table(int J, long long j0, double hstep, double kx, double ky, double kz,
                           double fc, double st, double* __restrict__ A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const double tc = hstep * (double)(j0 + j);
    const double inv2s2 = 1.0 / (2.0 * st * st);
    double acc = 0.0;
    for (int a = 0; a < NQ; ++a)
        for (int b = 0; b < NQ; ++b)
            for (int c = 0; c < NQ; ++c) {
                const double tau = tc - (c_qx[a] * kx + c_qx[b] * ky + c_qx[c] * kz);
                acc += c_qw[a] * c_qw[b] * c_qw[c] * sinpi(2.0 * fc * tau) * exp(-tau * tau * inv2s2);
            }
    A[j] = acc;
}

constexpr int kInterp = 10;   // interpolation points (degree 9)

__global__ void k_plane_wave_tab(long long M, int U, int V, const double* __restrict__ chi,
                                 double kx, double ky, double kz, double px, double py, double pz,
                                 double t0, int n_first, int n_steps, long long j0,
                                 double hstep, int J, const double* __restrict__ A,
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
    // position on the node lattice, and the distances to the 10 nodes around it, in
    // absolute node numbers (exact, and the same whichever call tabulated the nodes)
    const double xa = tc / hstep;
    long long ia = (long long)floor(xa) - (kInterp / 2 - 1);
    ia = min(max(ia, j0), j0 + J - kInterp);
    const double* Ai = A + (ia - j0);
    // barycentric weights of equispaced nodes: (-1)^j C(9, j)
    const double bw[kInterp] = {1.0, -9.0, 36.0, -84.0, 126.0, -126.0, 84.0, -36.0, 9.0, -1.0};
    double num = 0.0, den = 0.0, val = 0.0;
    bool hit = false;
#pragma unroll
    for (int j = 0; j < kInterp; ++j) {
        const double d = xa - (double)(ia + j);
        if (d == 0.0) { val = Ai[j]; hit = true; }
        const double c = bw[j] / d;
        num += c * Ai[j];
        den += c;
    }
    if (!hit) val = num / den;
    const double g = ch * val;
    o[0] = g * px;
    o[1] = g * py;
    o[2] = g * pz;
}

}  // namespace

namespace mot {

void excitation_setup(int dev) {
    // the __constant__ nodes live once per device and module: upload them the first
    // time a context is created on `dev` (a blocking copy, kept out of the per-call path)
    static std::mutex mu;
    static bool done[kMaxSetupDevices] = {};
    if (dev < 0 || dev >= kMaxSetupDevices)
        throw MotError{MOT_ERR_ARG, "device index beyond the supported range"};
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
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
    done[dev] = true;
}

void plane_wave(mot_ctx* c, const double k[3], const double p[3], double fc, double st, double t0,
                int n_first, int n_steps, double* Edev, cudaStream_t s) {
    if (!c->pw_tab) {   // no table buffer: the tensor rule at every voxel and step
        const long long tot = c->M * n_steps;
        k_plane_wave<<<(int)((tot + 255) / 256), 256, 0, s>>>(c->M, c->U, c->V, c->chi, k[0], k[1],
                                                              k[2], p[0], p[1], p[2], fc, st, t0,
                                                              n_first, n_steps, Edev);
        MOT_LAUNCH_CHECK();
        return;
    }
    // node spacing from the pulse's spectral extent; range of r_c . k_hat over the grid
    const double pi = 3.14159265358979323846;
    const double feff = std::fabs(fc) + 6.0 / (2.0 * pi * st);
    const double hstep = std::min(0.5, 0.057 / (2.0 * pi * feff));
    const int N[3] = {c->U, c->V, c->W};
    double rk_lo = 0.0, rk_hi = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e0 = 0.5 * k[a], e1 = (N[a] - 0.5) * k[a];
        rk_lo += std::min(e0, e1);
        rk_hi += std::max(e0, e1);
    }
    // steps per sub-call so that its tau range fits the table with 6 spare nodes a side
    const double span_rk = rk_hi - rk_lo;
    const int cap = (int)std::floor((kPwTable - 40) * hstep - span_rk);
    const int per = std::max(1, std::min(n_steps, cap));
    if (cap < 1) {      // a grid too large for one table even for one step
        const long long tot = c->M * n_steps;
        k_plane_wave<<<(int)((tot + 255) / 256), 256, 0, s>>>(c->M, c->U, c->V, c->chi, k[0], k[1],
                                                              k[2], p[0], p[1], p[2], fc, st, t0,
                                                              n_first, n_steps, Edev);
        MOT_LAUNCH_CHECK();
        return;
    }
    for (int s0 = 0; s0 < n_steps; s0 += per) {
        const int cnt = std::min(per, n_steps - s0);
        const int nf = n_first + s0;
        const double tlo = (double)nf - t0 - rk_hi, thi = (double)(nf + cnt - 1) - t0 - rk_lo;
        const long long j0 = (long long)std::floor(tlo / hstep) - 6;
        const int J = std::min(kPwTable, (int)((long long)std::ceil(thi / hstep) + 7 - j0));
        k_pw_table<<<(J + 127) / 128, 128, 0, s>>>(J, j0, hstep, k[0], k[1], k[2], fc, st,
                                                   c->pw_tab);
        MOT_LAUNCH_CHECK();
        const long long tot = c->M * cnt;
        k_plane_wave_tab<<<(int)((tot + 255) / 256), 256, 0, s>>>(
            c->M, c->U, c->V, c->chi, k[0], k[1], k[2], p[0], p[1], p[2], t0, nf, cnt, j0, hstep,
            J, c->pw_tab, Edev + (long long)s0 * 3 * c->M);
        MOT_LAUNCH_CHECK();
    }
}

}  // namespace mot

// Diagnostics of the stabilisation study (Sec. 6): the truncated MOT-JVIE of the
// finite-precision experiment, the FIR-regularisation magnitude (Eq. FIRmagnitude) and
// the tapered frequency response |H^alpha| of Eq. Halpha.
//
// Truncation: the finite-precision error epsilon of the interaction elements is
// estimated in Sec. 6 by deliberately truncating the element values to a step
// eps_trunc and watching when the per-step alternating solution changes.  Here every
// tabulated element G_l^{ab}(d) of a history lag l >= 1 is replaced by the nearest
// multiple of eps_trunc, and the spectra derived from the table are recomputed; the
// lag-0 elements (the Z_0 stencil of the per-step solve) are left as they are.
//
// Frequency response: the probe time series J_n = J(t_n), t_n = n dt, is tapered by a
// cosine window on its last fraction (the recommendation of Sec. 7.1 for a solution
// cut off while it still rings), transformed at the requested frequencies,
//     j(f) = dt sum_{n=1}^{N} w_n J_n exp(-2 pi i f t_n),
// and divided by eps0 (eps_r - 1) |e^i(f)| with the amplitude spectrum of the
// modulated Gaussian incident pulse sin(2 pi f_c tau) exp(-tau^2 / (2 sigma_t^2)),
//     |e^i(f)| = sigma_t sqrt(2 pi) / 2 |exp(-2 pi^2 sigma_t^2 (f - f_c)^2)
//                                     - exp(-2 pi^2 sigma_t^2 (f + f_c)^2)|
// (units eps0 = c0 = 1).
#include "mot_internal.cuh"

#include <cmath>
#include <new>
#include <vector>

namespace {

constexpr int NT = 256;

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// tab[o][cc][k] (lag tab_l0[o] + k) -> nearest multiple of q for lags >= 1
__global__ void k_truncate(const int* __restrict__ tab_l0, double* __restrict__ tab,
                           long long noff, double q) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= noff * 6 * mot::WIN) return;
    const long long o = i / (6 * mot::WIN);
    const int k = (int)(i % mot::WIN);
    if (tab_l0[o] + k >= 1) tab[i] = q * rint(tab[i] / q);
}

// one thread per (frequency, probe, component): tapered DFT of the probe series
__global__ void k_tapered_dft(const double* __restrict__ J, int n_steps, int n_probe,
                              double dt, int n_flat, const double* __restrict__ freqs,
                              int n_freq, double2* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_f = 3LL * n_probe;
    if (i >= per_f * n_freq) return;
    const int f = (int)(i / per_f);
    const long long pa = i % per_f;          // probe * 3 + component
    const double fr = freqs[f];
    const int n_taper = n_steps - n_flat;
    double re = 0.0, im = 0.0;
    for (int n = 1; n <= n_steps; ++n) {
        double w = 1.0;
        if (n > n_flat) w = 0.5 * (1.0 + cospi((double)(n - n_flat) / (double)n_taper));
        // exp(-2 pi i f t_n): reduce f n dt modulo 1 before the sine and cosine
        double ph = fr * dt * (double)n;
        ph -= floor(ph);
        double s, c;
        sincospi(2.0 * ph, &s, &c);
        const double v = w * J[(long long)(n - 1) * per_f + pa];
        re = fma(v, c, re);
        im = fma(-v, s, im);
    }
    out[i] = make_double2(dt * re, dt * im);
}

__global__ void k_response(const double2* __restrict__ jf, int n_probe,
                           const double* __restrict__ eps_probe, const double* __restrict__ freqs,
                           int n_freq, double f_c, double sigma_t, double* __restrict__ H) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_f = 3LL * n_probe;
    if (i >= per_f * n_freq) return;
    const int f = (int)(i / per_f);
    const int p = (int)((i % per_f) / 3);
    const double fr = freqs[f];
    const double g = 2.0 * M_PI * M_PI * sigma_t * sigma_t;
    const double ei = sigma_t * sqrt(2.0 * M_PI) * 0.5 *
                      fabs(exp(-g * (fr - f_c) * (fr - f_c)) - exp(-g * (fr + f_c) * (fr + f_c)));
    const double2 v = jf[i];
    H[i] = hypot(v.x, v.y) / ((eps_probe[p] - 1.0) * ei);
}

bool device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

mot_status mot_truncate_table(mot_ctx* c, double eps_trunc) {
    if (!c) return MOT_ERR_ARG;
    if (c->shared_src || c->n_shared) {
        c->err = "mot_truncate_table: the table of a shared setup cannot change";
        return MOT_ERR_ARG;
    }
    if (c->n_done || c->adj_total) {
        c->err = "mot_truncate_table: call before the first step";
        return MOT_ERR_ARG;
    }
    if (!(eps_trunc > 0.0) || !std::isfinite(eps_trunc)) {
        c->err = "mot_truncate_table: eps_trunc must be finite and > 0";
        return MOT_ERR_ARG;
    }
    if (c->broken) return MOT_ERR_STATE;
    try {
        const long long noff = (long long)c->U * c->V * c->W;
        k_truncate<<<nblk(noff * 6 * mot::WIN, NT), NT, 0, c->stream>>>(c->tab_l0, c->tab, noff,
                                                                        eps_trunc);
        MOT_LAUNCH_CHECK();
        mot::compute_spectra(c);
        if (c->scheme == MOT_HISTORY_BLOCKED) {
            if (c->precision == MOT_FP64) mot::level_spectra<double>(c);
            else mot::level_spectra<float>(c);
        }
        c->pdsa_n = c->pdsa_flags = -1;
        MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
        return MOT_OK;
    } catch (const MotError& e) {
        c->err = e.msg;
        if (e.st == MOT_ERR_CUDA) c->broken = true;
        return e.st;
    }
}

mot_status mot_fir_magnitude(const double* taps, int n_taps, int n_theta, const double* theta,
                             double* out) {
    if (n_taps < 0 || n_theta < 0 || (n_taps && !taps) || (n_theta && (!theta || !out)))
        return MOT_ERR_ARG;
    for (int t = 0; t < n_theta; ++t) {
        double re = 0.0, im = 0.0;
        for (int n = 0; n < n_taps; ++n) {
            re += taps[n] * std::cos(n * theta[t]);
            im -= taps[n] * std::sin(n * theta[t]);
        }
        out[t] = std::hypot(re, im);
    }
    return MOT_OK;
}

mot_status mot_frequency_response(int n_steps, int n_probe, const double* J, double dt,
                                  double taper, const double* eps_probe, double f_c,
                                  double sigma_t, int n_freq, const double* freqs, double* H,
                                  double* j_hat) {
    if (n_steps < 1 || n_probe < 1 || n_freq < 1 || !J || !eps_probe || !freqs || !H ||
        !(dt > 0.0) || !(taper >= 0.0 && taper < 1.0) || !(sigma_t > 0.0))
        return MOT_ERR_ARG;
    for (int p = 0; p < n_probe; ++p)
        if (!(eps_probe[p] > 1.0)) return MOT_ERR_ARG;
    const long long nJ = (long long)n_steps * n_probe * 3;
    const long long nO = (long long)n_freq * n_probe * 3;
    double *dJ = nullptr, *de = nullptr, *df = nullptr, *dH = nullptr;
    double2* dj = nullptr;
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e) { if (err == cudaSuccess) err = e; };
    const bool jdev = device_ptr(J);
    if (!jdev) chk(cudaMalloc(&dJ, sizeof(double) * nJ));
    chk(cudaMalloc(&de, sizeof(double) * n_probe));
    chk(cudaMalloc(&df, sizeof(double) * n_freq));
    chk(cudaMalloc(&dH, sizeof(double) * nO));
    chk(cudaMalloc(&dj, sizeof(double2) * nO));
    if (err == cudaSuccess) {
        if (!jdev) chk(cudaMemcpy(dJ, J, sizeof(double) * nJ, cudaMemcpyHostToDevice));
        chk(cudaMemcpy(de, eps_probe, sizeof(double) * n_probe, cudaMemcpyHostToDevice));
        chk(cudaMemcpy(df, freqs, sizeof(double) * n_freq, cudaMemcpyHostToDevice));
    }
    if (err == cudaSuccess) {
        // samples n <= n_flat keep weight 1; the last fraction `taper` falls off as a
        // half cosine to 0 at n = N
        const int n_flat = n_steps - (int)std::floor(taper * n_steps);
        k_tapered_dft<<<nblk(nO, NT), NT>>>(jdev ? J : dJ, n_steps, n_probe, dt, n_flat, df,
                                             n_freq, dj);
        chk(cudaGetLastError());
        k_response<<<nblk(nO, NT), NT>>>(dj, n_probe, de, df, n_freq, f_c, sigma_t, dH);
        chk(cudaGetLastError());
        chk(cudaMemcpy(H, dH, sizeof(double) * nO, cudaMemcpyDeviceToHost));
        if (j_hat) chk(cudaMemcpy(j_hat, dj, sizeof(double2) * nO, cudaMemcpyDeviceToHost));
    }
    cudaFree(dJ);
    cudaFree(de);
    cudaFree(df);
    cudaFree(dH);
    cudaFree(dj);
    if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? MOT_ERR_OOM : MOT_ERR_CUDA;
    return MOT_OK;
}

}  // extern "C"

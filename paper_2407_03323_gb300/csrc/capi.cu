// C ABI of the marching library: context lifetime, excitation staging and the step
// loop (Eqs. MOTInversion, PnMOT).  Per step n:
//   1. forward FFT of J_{n-1} into the spectral ring        (Sec. 3)
//   2. lag MAC over the ring, inverse FFT -> (G * J)_hist    (Eq. PnFFTMOT)
//   3. FIR epilogue -> rhs, CG solve of Z_0 J_n = rhs        (Eq. MOTInversion, Sec. 6.1)
//   4. ||J_n|| monitor, optional AoS write-out
#include "mot_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

namespace {

thread_local std::string g_create_error;

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool smooth7(int n) {
    for (int r : {2, 3, 5, 7})
        while (n % r == 0) n /= r;
    return n == 1;
}

int pad_size(int N) {
    int P = std::max(2 * N - 1, 2);
    while (P % 2 != 0 || !smooth7(P)) ++P;
    return P;
}

template <typename F>
mot_status guarded(mot_ctx* c, F&& f) {
    if (c && c->broken) return MOT_ERR_STATE;
    try {
        f();
        return MOT_OK;
    } catch (const MotError& e) {
        if (c) {
            c->err = e.msg;
            if (e.st == MOT_ERR_CUDA || e.st == MOT_ERR_TIMEOUT) c->broken = true;
        }
        return e.st;
    } catch (const std::bad_alloc&) {
        if (c) c->err = "host allocation failed";
        return MOT_ERR_OOM;
    }
}

template <typename R> void alloc_history(mot_ctx* c) { mot::history_alloc<R>(c); }

void free_all(mot_ctx* c) {
    cudaFree(c->adj_gchi);
    c->adj_gchi = nullptr;
    if (c->shared_src) {   // borrowed setup: release the references, free the state only
        for (int a = 0; a < 3; ++a) c->ax[a] = AxisFFT();
        for (int k = 0; k < 8; ++k) c->lev_fft[k] = AxisFFT();
        c->eps = c->chi = c->cg_diag = c->tab = nullptr;
        c->vfac = nullptr;
        c->tab_l0 = nullptr;
        c->active = c->nmask = c->tiles = nullptr;
        c->diag32 = nullptr;
        c->h64.ghat = nullptr; c->h64.level_spec = nullptr;
        c->h32.ghat = nullptr; c->h32.level_spec = nullptr;
        c->shared_src->n_shared -= 1;
        c->shared_src = nullptr;
    }
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    for (int a = 0; a < 3; ++a) mot::fft_free_axis(c->ax[a]);
    for (int k = 0; k < 8; ++k) mot::fft_free_axis(c->lev_fft[k]);
    mot::history_free<double>(c);
    mot::history_free<float>(c);
    double* dptrs[] = {c->eps, c->chi, c->cg_diag, c->J, c->rhs, c->cg_r,
                       c->cg_q, c->red, c->norms, c->outbuf, c->tab, c->Estage};
    for (double* p : dptrs) cudaFree(p);
    cudaFree(c->tab_l0);
    cudaFree(c->dstatus);
    cudaFree(c->cg32);
    cudaFree(c->cg_df);
    cudaFree(c->active);
    cudaFree(c->nmask);
    cudaFree(c->tiles);
    cudaFree(c->diag32);
    cudaFree(c->vfac);
    cudaFree(c->probe_tab);
    cudaFree(c->probe_l0);
    cudaFree(c->pdsa_spec);
    cudaFree(c->pdsa_a);
    cudaFree(c->pdsa_xhat);
    cudaFree(c->pdsa_conv);
    cudaFree(c->pw_tab);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    c->events.clear();
    for (cudaEvent_t e : c->e_chunk) cudaEventDestroy(e);
    c->e_chunk.clear();
    for (int k = 0; k < 3; ++k) {
        if (c->out_ready[k]) cudaEventDestroy(c->out_ready[k]);
        if (c->out_done[k]) cudaEventDestroy(c->out_done[k]);
    }
    if (c->cstream) cudaStreamDestroy(c->cstream);
    if (c->hstream) cudaStreamDestroy(c->hstream);
    if (c->stream) cudaStreamDestroy(c->stream);
}

void reset_state(mot_ctx* c, cudaStream_t s) {
    MOT_CUDA_TRY(cudaMemsetAsync(c->J, 0, sizeof(double) * 3 * c->M * c->jring, s));
    if (c->precision == MOT_FP64) mot::history_reset<double>(c, s);
    else mot::history_reset<float>(c, s);
    c->n_done = 0;
    c->E_count = 0;
    c->peak_norm = 0.0;
    c->last_norm = 0.0;
    c->fail_step = 0;
}

void history_for(mot_ctx* c, int n, cudaStream_t s, cudaEvent_t* ev = nullptr) {
    if (c->precision == MOT_FP64) mot::history_step<double>(c, n, s, ev);
    else mot::history_step<float>(c, n, s, ev);
}

constexpr int kOutSlots = 3;   // output ring depth (host J_out)

void ensure_copy_stream(mot_ctx* c) {
    if (!c->cstream) MOT_CUDA_TRY(cudaStreamCreateWithFlags(&c->cstream, cudaStreamNonBlocking));
}

void ensure_stage_stream(mot_ctx* c) {
    if (!c->hstream) MOT_CUDA_TRY(cudaStreamCreateWithFlags(&c->hstream, cudaStreamNonBlocking));
}

cudaEvent_t new_sync_event() {
    cudaEvent_t e;
    MOT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return e;
}

void ensure_events(mot_ctx* c, size_t n) {
    while (c->events.size() < n) {
        cudaEvent_t e;
        MOT_CUDA_TRY(cudaEventCreate(&e));
        c->events.push_back(e);
    }
}

}  // namespace

extern "C" {

mot_status mot_create(const int grid[3], const double h[3], double dt, const double* eps_r,
                      const double* fir_taps, int n_taps, int precision, int scheme, int block,
                      mot_ctx** out) {
    return mot_create_padded(grid, h, dt, eps_r, fir_taps, n_taps, precision, scheme, block,
                             nullptr, out);
}

mot_status mot_create_padded(const int grid[3], const double h[3], double dt,
                             const double* eps_r, const double* fir_taps, int n_taps,
                             int precision, int scheme, int block, const int fft_len[3],
                             mot_ctx** out) {
    if (out) *out = nullptr;
    g_create_error.clear();
    auto fail = [](mot_status st, const std::string& m) {
        g_create_error = m;
        return st;
    };
    if (!grid || !h || !eps_r || !out) return fail(MOT_ERR_ARG, "null argument");
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 1 || grid[a] > 1024) return fail(MOT_ERR_ARG, "grid sizes must be in 1..1024");
    if ((long long)grid[0] * grid[1] * grid[2] > (1LL << 30))
        return fail(MOT_ERR_ARG, "at most 2^30 voxels");
    if (!(h[0] > 0) || h[0] != h[1] || h[0] != h[2])
        return fail(MOT_ERR_ARG, "voxels must be cubes (h[0] == h[1] == h[2] > 0)");
    if (!(dt > 0) || std::fabs(dt - h[0]) > 1e-12 * h[0])
        return fail(MOT_ERR_ARG, "the element quadrature requires c0 dt == h (c0 = 1)");
    if (n_taps < 0 || n_taps > 64 || (n_taps > 0 && !fir_taps))
        return fail(MOT_ERR_ARG, "n_taps must be 0..64 and fir_taps non-null when n_taps > 0");
    if (precision != MOT_FP64 && precision != MOT_FP32_HISTORY)
        return fail(MOT_ERR_ARG, "unknown precision");
    if (scheme != MOT_HISTORY_DIRECT && scheme != MOT_HISTORY_BLOCKED &&
        scheme != MOT_HISTORY_BLOCKED_DOUBLING)
        return fail(MOT_ERR_ARG, "unknown history scheme");
    if (scheme != MOT_HISTORY_DIRECT && (block < 2 || (block & (block - 1)) != 0))
        return fail(MOT_ERR_ARG, "block must be a power of two >= 2 for the blocked scheme");
    if (fft_len)
        for (int a = 0; a < 3; ++a)
            if (fft_len[a] < std::max(2 * grid[a] - 1, 2) || fft_len[a] > 4096 ||
                fft_len[a] % 2 != 0 || !smooth7(fft_len[a]))
                return fail(MOT_ERR_ARG, "fft_len[a] must be even, 7-smooth, >= 2 grid[a] - 1 "
                                         "and <= 4096");
    const long long M = (long long)grid[0] * grid[1] * grid[2];
    for (long long m = 0; m < M; ++m)
        if (!(eps_r[m] >= 1.0) || !std::isfinite(eps_r[m]))
            return fail(MOT_ERR_ARG, "eps_r must be finite and >= 1");

    mot_ctx* c = new (std::nothrow) mot_ctx();
    if (!c) return fail(MOT_ERR_OOM, "host allocation failed");
    c->U = grid[0]; c->V = grid[1]; c->W = grid[2];
    c->M = M;
    c->precision = precision;
    // both blocked plans run the same code; they differ in the last level only
    c->scheme = scheme == MOT_HISTORY_DIRECT ? MOT_HISTORY_DIRECT : MOT_HISTORY_BLOCKED;
    c->lev_fit = scheme == MOT_HISTORY_BLOCKED;
    c->block = block;
    c->n_taps = n_taps;
    c->taps.assign(fir_taps, fir_taps + n_taps);
    // per-step solve tolerance: the FP32-history variant's history P carries ~2e-7
    // relative error per step (FP32 FFT convolution), so a residual of 3e-8 ||rhs/chi||
    // stays below it (the FP32-vs-FP64 deviation of the march is the same for 1e-10 ..
    // 3e-8); FP64 solves to 1e-13
    c->tol = precision == MOT_FP64 ? 1e-13 : 3e-8;
    // Eq. Ell with h = c dt = 1
    c->ell = (int)std::floor(std::sqrt((double)c->U * c->U + (double)c->V * c->V +
                                       (double)c->W * c->W)) + 2;
    mot_status st = guarded(c, [&] {
        int dev = 0;
        MOT_CUDA_TRY(cudaGetDevice(&dev));
        c->device = dev;
        MOT_CUDA_TRY(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev));
        mot::excitation_setup(dev);
        MOT_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        const int N[3] = {c->U, c->V, c->W};
        for (int a = 0; a < 3; ++a)
            mot::fft_plan_axis(c->ax[a], fft_len ? fft_len[a] : pad_size(N[a]));
        c->Hu = c->ax[0].P / 2 + 1;
        c->Hv = c->ax[1].P / 2 + 1;
        c->Hw = c->ax[2].P / 2 + 1;
        c->nbins = (long long)c->ax[2].P * c->ax[1].P * c->Hu;
        c->noct = (long long)c->Hw * c->Hv * c->Hu;
        // geometry
        std::vector<double> e(eps_r, eps_r + M), chi(M), dg(M);
        const double d0 = n_taps > 0 ? fir_taps[0] : 0.0;
        for (long long m = 0; m < M; ++m) {
            chi[m] = (e[m] - 1.0) / e[m];
            dg[m] = chi[m] > 0.0 ? (0.5 / e[m] + d0) / chi[m] : 0.0;
        }
        MOT_CUDA_TRY(cudaMalloc(&c->eps, sizeof(double) * M));
        MOT_CUDA_TRY(cudaMalloc(&c->chi, sizeof(double) * M));
        MOT_CUDA_TRY(cudaMalloc(&c->cg_diag, sizeof(double) * M));
        MOT_CUDA_TRY(cudaMemcpy(c->eps, e.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
        MOT_CUDA_TRY(cudaMemcpy(c->chi, chi.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
        MOT_CUDA_TRY(cudaMemcpy(c->cg_diag, dg.data(), sizeof(double) * M, cudaMemcpyHostToDevice));
        // elements, stencil, spectra
        mot::compute_table(c);
        mot::stencil_setup(c);
        if (precision == MOT_FP64) alloc_history<double>(c);
        else alloc_history<float>(c);
        mot::compute_spectra(c);
        if (c->scheme == MOT_HISTORY_BLOCKED) {
            if (precision == MOT_FP64) mot::level_spectra<double>(c);
            else mot::level_spectra<float>(c);
        }
        // marching state
        c->jring = std::max(n_taps, 4) + 1;
        MOT_CUDA_TRY(cudaMalloc(&c->J, sizeof(double) * 3 * M * c->jring));
        MOT_CUDA_TRY(cudaMalloc(&c->rhs, sizeof(double) * 3 * M));
        MOT_CUDA_TRY(cudaMalloc(&c->cg_r, sizeof(double) * 3 * M));
        MOT_CUDA_TRY(cudaMalloc(&c->cg_q, sizeof(double) * 3 * M));
        MOT_CUDA_TRY(cudaMalloc(&c->cg32, sizeof(float) * 16 * M));
        MOT_CUDA_TRY(cudaMemset(c->cg32, 0, sizeof(float) * 16 * M));
        {
            std::vector<int> act, nm;
            for (long long m = 0; m < M; ++m) {
                if (!(chi[m] > 0.0)) continue;
                act.push_back((int)m);
                const int u = (int)(m % c->U), v = (int)((m / c->U) % c->V),
                          w = (int)(m / ((long long)c->U * c->V));
                int mask = 0;
                for (int ez = -1; ez <= 1; ++ez)
                    for (int ey = -1; ey <= 1; ++ey)
                        for (int ex = -1; ex <= 1; ++ex) {
                            const bool in = u + ex >= 0 && u + ex < c->U && v + ey >= 0 &&
                                            v + ey < c->V && w + ez >= 0 && w + ez < c->W;
                            if (in) mask |= 1 << ((ez + 1) * 9 + (ey + 1) * 3 + (ex + 1));
                        }
                nm.push_back(mask);
            }
            c->nact = (long long)act.size();
            const size_t na = std::max<size_t>(act.size(), 1);
            MOT_CUDA_TRY(cudaMalloc(&c->active, sizeof(int) * na));
            MOT_CUDA_TRY(cudaMalloc(&c->nmask, sizeof(int) * na));
            if (c->nact) {
                MOT_CUDA_TRY(cudaMemcpy(c->active, act.data(), sizeof(int) * c->nact,
                                        cudaMemcpyHostToDevice));
                MOT_CUDA_TRY(cudaMemcpy(c->nmask, nm.data(), sizeof(int) * c->nact,
                                        cudaMemcpyHostToDevice));
            }
            {   // 8^3 tiles that hold at least one active voxel
                std::vector<int> tl;
                for (int z0 = 0; z0 < c->W; z0 += 8)
                    for (int y0 = 0; y0 < c->V; y0 += 8)
                        for (int x0 = 0; x0 < c->U; x0 += 8) {
                            bool any = false;
                            for (int z = z0; z < std::min(z0 + 8, c->W) && !any; ++z)
                                for (int y = y0; y < std::min(y0 + 8, c->V) && !any; ++y)
                                    for (int x = x0; x < std::min(x0 + 8, c->U) && !any; ++x)
                                        any = chi[((long long)z * c->V + y) * c->U + x] > 0.0;
                            if (any) tl.push_back(x0 | (y0 << 10) | (z0 << 20));
                        }
                c->ntiles = (int)tl.size();
                // one block per tile at most: the tiled passes give a block one tile at
                // a time, so further blocks would only wait at the grid barriers (and
                // keep SMs from concurrent solves of other contexts)
                c->cg_blocks = std::min(c->cg_blocks, std::max(c->ntiles, 1));
                MOT_CUDA_TRY(cudaMalloc(&c->tiles, sizeof(int) * std::max<size_t>(tl.size(), 1)));
                if (!tl.empty())
                    MOT_CUDA_TRY(cudaMemcpy(c->tiles, tl.data(), sizeof(int) * tl.size(),
                                            cudaMemcpyHostToDevice));
            }
            std::vector<float> d32(M);
            std::vector<double> vf(4 * M);
            for (long long m = 0; m < M; ++m) {
                d32[m] = (float)dg[m];
                vf[m] = 0.5 / e[m];
                vf[M + m] = chi[m] > 0.0 ? 1.0 / chi[m] : 0.0;
                vf[2 * M + m] = 1.0 / (0.5 / e[m] + d0);
                vf[3 * M + m] = chi[m];
            }
            MOT_CUDA_TRY(cudaMalloc(&c->diag32, sizeof(float) * M));
            MOT_CUDA_TRY(cudaMalloc(&c->vfac, sizeof(double) * 4 * M));
            MOT_CUDA_TRY(cudaMemcpy(c->diag32, d32.data(), sizeof(float) * M, cudaMemcpyHostToDevice));
            if (precision == MOT_FP32_HISTORY) {
                // float-pair state of the double-float residual; entries of inactive
                // voxels stay zero (neighbours read them)
                MOT_CUDA_TRY(cudaMalloc(&c->cg_df, sizeof(float) * 17 * M));
                MOT_CUDA_TRY(cudaMemset(c->cg_df, 0, sizeof(float) * 16 * M));
                std::vector<float> dlo(M);
                for (long long m = 0; m < M; ++m) dlo[m] = (float)(dg[m] - (double)d32[m]);
                MOT_CUDA_TRY(cudaMemcpy(c->cg_df + 16 * M, dlo.data(), sizeof(float) * M,
                                        cudaMemcpyHostToDevice));
            }
            MOT_CUDA_TRY(cudaMemcpy(c->vfac, vf.data(), sizeof(double) * 4 * M, cudaMemcpyHostToDevice));
        }
        MOT_CUDA_TRY(cudaMalloc(&c->red, sizeof(double) * 3 * std::max(c->cg_blocks, 1)));
        if (c->nact) mot::chebyshev_setup(c);
        MOT_CUDA_TRY(cudaMalloc(&c->dstatus, sizeof(int) * mot::kStatusWords));
        MOT_CUDA_TRY(cudaMemset(c->dstatus, 0, sizeof(int) * mot::kStatusWords));
        MOT_CUDA_TRY(cudaMalloc(&c->pw_tab, sizeof(double) * mot::kPwTable));
        reset_state(c, c->stream);
        MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    });
    if (st != MOT_OK) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return MOT_OK;
}

void mot_destroy(mot_ctx* c) {
    if (!c || c->rhs_owner) return;   // a right-hand side goes with the context owning it
    cudaDeviceSynchronize();
    for (mot_ctx* r : c->rhs_ctx) {   // they borrow this context's setup
        free_all(r);
        delete r;
    }
    c->rhs_ctx.clear();
    free_all(c);
    delete c;
}

mot_status mot_create_shared(mot_ctx* src, mot_ctx** out) {
    if (!out) return MOT_ERR_ARG;
    *out = nullptr;
    if (!src) { g_create_error = "source context is NULL"; return MOT_ERR_ARG; }
    if (src->broken) return MOT_ERR_STATE;
    if (src->shared_src) { src = src->shared_src; }   // share the owner of the setup
    mot_ctx* c = new mot_ctx();
    // grid, discretisation and solver setup (values), shared device setup (pointers)
    c->U = src->U; c->V = src->V; c->W = src->W; c->M = src->M; c->ell = src->ell;
    for (int a = 0; a < 3; ++a) c->ax[a] = src->ax[a];
    c->Hu = src->Hu; c->Hv = src->Hv; c->Hw = src->Hw;
    c->nbins = src->nbins; c->noct = src->noct;
    c->precision = src->precision; c->scheme = src->scheme; c->block = src->block;
    c->n_taps = src->n_taps; c->taps = src->taps;
    c->tol = src->tol; c->max_iter = src->max_iter; c->growth = src->growth;
    c->jring = src->jring; c->hring = src->hring;
    c->eps = src->eps; c->chi = src->chi; c->cg_diag = src->cg_diag;
    c->active = src->active; c->nmask = src->nmask; c->tiles = src->tiles;
    c->ntiles = src->ntiles; c->nact = src->nact;
    c->diag32 = src->diag32; c->vfac = src->vfac;
    c->cheb_lmin = src->cheb_lmin; c->cheb_lmax = src->cheb_lmax; c->cheb_n = src->cheb_n;
    c->cheb_log_rate = src->cheb_log_rate; c->cheb_inv_theta = src->cheb_inv_theta;
    for (int k = 0; k < 64; ++k) { c->cheb_c1[k] = src->cheb_c1[k]; c->cheb_c2[k] = src->cheb_c2[k]; }
    for (int k = 0; k < 27 * 6; ++k) c->stencil[k] = src->stencil[k];
    for (int e = 0; e < 27; ++e) c->noff[e] = src->noff[e];
    c->tab_l0 = src->tab_l0; c->tab = src->tab;
    c->nlev = src->nlev;
    c->lev_period = src->lev_period;
    c->lev_fit = src->lev_fit;
    for (int k = 0; k < 8; ++k) {
        c->lev_S[k] = src->lev_S[k]; c->lev_a[k] = src->lev_a[k]; c->lev_off[k] = src->lev_off[k];
        c->lev_fft[k] = src->lev_fft[k]; c->lev_acc[k] = src->lev_acc[k];
    }
    c->smax = src->smax;
    c->nsm = src->nsm; c->cg_blocks = src->cg_blocks; c->bar_budget = src->bar_budget;
    c->device = src->device;
    c->shared_src = src;
    src->n_shared += 1;
    const long long M = c->M;
    mot_status st = guarded(c, [&] {
        MOT_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        if (c->precision == MOT_FP64) mot::history_alloc_shared<double>(c, src);
        else mot::history_alloc_shared<float>(c, src);
        MOT_CUDA_TRY(cudaMalloc(&c->J, sizeof(double) * 3 * M * c->jring));
        MOT_CUDA_TRY(cudaMalloc(&c->rhs, sizeof(double) * 3 * M));
        MOT_CUDA_TRY(cudaMalloc(&c->cg_r, sizeof(double) * 3 * M));
        MOT_CUDA_TRY(cudaMalloc(&c->cg_q, sizeof(double) * 3 * M));
        MOT_CUDA_TRY(cudaMalloc(&c->cg32, sizeof(float) * 16 * M));
        MOT_CUDA_TRY(cudaMemset(c->cg32, 0, sizeof(float) * 16 * M));
        if (src->cg_df) {
            MOT_CUDA_TRY(cudaMalloc(&c->cg_df, sizeof(float) * 17 * M));
            MOT_CUDA_TRY(cudaMemset(c->cg_df, 0, sizeof(float) * 16 * M));
            MOT_CUDA_TRY(cudaMemcpy(c->cg_df + 16 * M, src->cg_df + 16 * M, sizeof(float) * M,
                                    cudaMemcpyDeviceToDevice));
        }
        MOT_CUDA_TRY(cudaMalloc(&c->red, sizeof(double) * 3 * std::max(c->cg_blocks, 1)));
        MOT_CUDA_TRY(cudaMalloc(&c->dstatus, sizeof(int) * mot::kStatusWords));
        MOT_CUDA_TRY(cudaMemset(c->dstatus, 0, sizeof(int) * mot::kStatusWords));
        MOT_CUDA_TRY(cudaMalloc(&c->pw_tab, sizeof(double) * mot::kPwTable));
        reset_state(c, c->stream);
        MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    });
    if (st != MOT_OK) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return MOT_OK;
}

mot_status mot_set_excitation(mot_ctx* c, int n_steps, const double* E, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (n_steps < 1 || !E) { c->err = "n_steps >= 1 and E non-null required"; return MOT_ERR_ARG; }
    return guarded(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        if (c->hstream) {   // a host staging still in flight writes the buffer: order after it
            cudaEvent_t pending = new_sync_event();
            MOT_CUDA_TRY(cudaEventRecord(pending, c->hstream));
            MOT_CUDA_TRY(cudaStreamWaitEvent(s, pending, 0));
            cudaEventDestroy(pending);
        }
        if (n_steps > c->E_cap) {
            MOT_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(c->Estage);
            c->Estage = nullptr;
            c->E_cap = 0;
            MOT_CUDA_TRY(cudaMalloc(&c->Estage, sizeof(double) * 3 * c->M * n_steps));
            c->E_cap = n_steps;
        }
        const long long step = 3 * c->M;
        if (is_device_ptr(E)) {
            MOT_CUDA_TRY(cudaMemcpyAsync(c->Estage, E, sizeof(double) * step * n_steps,
                                         cudaMemcpyDeviceToDevice, s));
            c->e_chunk_steps = 0;
        } else {
            // host source: chunks of ~64 MB on the staging stream, each with an event, so
            // that mot_march starts on the first steps while the rest still arrives;
            // the copies wait for work already queued on s (it may read the buffer)
            ensure_stage_stream(c);
            const int ch = (int)std::max(1LL, (64LL << 20) / (long long)(sizeof(double) * step));
            const int nch = (n_steps + ch - 1) / ch;
            while ((int)c->e_chunk.size() < nch) c->e_chunk.push_back(new_sync_event());
            cudaEvent_t before = new_sync_event();
            MOT_CUDA_TRY(cudaEventRecord(before, s));
            MOT_CUDA_TRY(cudaStreamWaitEvent(c->hstream, before, 0));
            cudaEventDestroy(before);
            for (int j = 0; j < nch; ++j) {
                const long long a = (long long)j * ch, b = std::min<long long>(n_steps, a + ch);
                MOT_CUDA_TRY(cudaMemcpyAsync(c->Estage + a * step, E + a * step,
                                             sizeof(double) * step * (b - a),
                                             cudaMemcpyHostToDevice, c->hstream));
                MOT_CUDA_TRY(cudaEventRecord(c->e_chunk[j], c->hstream));
            }
            c->e_chunk_steps = ch;
        }
        c->E_first = c->n_done + 1;
        c->E_count = n_steps;
    });
}

mot_status mot_plane_wave(mot_ctx* c, const double k_hat[3], const double p_hat[3], double f_c,
                          double sigma_t, double t0, int n_first, int n_steps, double* E_out,
                          void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (!k_hat || !p_hat || !E_out || n_steps < 1 || !(sigma_t > 0)) {
        c->err = "invalid plane-wave arguments";
        return MOT_ERR_ARG;
    }
    return guarded(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        if (is_device_ptr(E_out)) {
            mot::plane_wave(c, k_hat, p_hat, f_c, sigma_t, t0, n_first, n_steps, E_out, s);
        } else {
            double* tmp = nullptr;
            MOT_CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * 3 * c->M * n_steps));
            try {
                mot::plane_wave(c, k_hat, p_hat, f_c, sigma_t, t0, n_first, n_steps, tmp, s);
                MOT_CUDA_TRY(cudaMemcpyAsync(E_out, tmp, sizeof(double) * 3 * c->M * n_steps,
                                             cudaMemcpyDeviceToHost, s));
                MOT_CUDA_TRY(cudaStreamSynchronize(s));
            } catch (...) {
                cudaFree(tmp);
                throw;
            }
            cudaFree(tmp);
        }
    });
}

}  // extern "C"

namespace {

// Capture the launches of `launch_period` (one period of the march) on s into a graph,
// update the context's executable graph in place with its arguments (the kernels and
// their order are the same every period; ring slots, step indices, the excitation and
// output pointers change), instantiate it on the first period or when the update is
// refused, and launch it.  Launches already enqueued keep the arguments they had.
template <typename F>
void march_period_graph(mot_ctx* c, cudaStream_t s, F&& launch_period) {
    cudaGraph_t g = nullptr;
    MOT_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
        launch_period();
    } catch (...) {
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
    }
    MOT_CUDA_TRY(cudaStreamEndCapture(s, &g));
    struct Guard {
        cudaGraph_t g;
        ~Guard() { cudaGraphDestroy(g); }
    } guard{g};
    if (c->gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
    }
    if (!c->gexec) {
        MOT_CUDA_TRY(cudaGraphInstantiate(&c->gexec, g, 0));
        c->stats.graph_instantiations += 1;
    }
    MOT_CUDA_TRY(cudaGraphLaunch(c->gexec, s));
    c->stats.graph_launches += 1;
}

// One mot_march call on one context, in stages so that several contexts (the
// right-hand sides of mot_march_rhs) can interleave their launches: begin() sizes the
// buffers and clears the device status; launch_step(i) / launch_all() enqueue the
// steps on the context's stream; fetch() waits for the stream, reads the per-step
// norms and the solve's status words and applies the stability monitor (Sec. 5.2).
struct MarchRun {
    mot_ctx* c;
    int n_steps;
    double* J_out;
    cudaStream_t s;
    bool dev_out = false, graphs = false, graphs_allowed = true;
    int waited_chunk = -1;
    long long step = 0;
    mot_status result = MOT_OK;

    void begin() {
        dev_out = is_device_ptr(J_out);
        if (n_steps > c->norms_cap) {
            MOT_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(c->norms);
            c->norms = nullptr;
            c->norms_cap = 0;
            MOT_CUDA_TRY(cudaMalloc(&c->norms, sizeof(double) * n_steps));
            c->norms_cap = n_steps;
        }
        step = 3 * c->M;
        if (J_out && !dev_out) {
            if (!c->outbuf) MOT_CUDA_TRY(cudaMalloc(&c->outbuf, sizeof(double) * step * kOutSlots));
            ensure_copy_stream(c);
            for (int k = 0; k < kOutSlots; ++k) {
                if (!c->out_ready[k]) c->out_ready[k] = new_sync_event();
                if (!c->out_done[k]) c->out_done[k] = new_sync_event();
            }
        }
        MOT_CUDA_TRY(cudaMemsetAsync(c->dstatus, 0, sizeof(int) * mot::kStatusWords, s));
        if (c->profiling) ensure_events(c, 6 * (size_t)n_steps);
        // whole periods as one CUDA graph: device-resident excitation and outputs, no
        // per-phase events, a capturable stream
        graphs = graphs_allowed && c->graph_steps > 0 && !c->profiling && (!J_out || dev_out) &&
                 s != cudaStreamLegacy && s != cudaStreamPerThread && s != nullptr;
        if (graphs && c->e_chunk_steps > 0)   // the whole staged excitation, before capture
            for (cudaEvent_t e : c->e_chunk) MOT_CUDA_TRY(cudaStreamWaitEvent(s, e, 0));
    }

    void launch_step(int i) {
        const int n = c->n_done + 1 + i;
        const double* En = nullptr;
        if (c->E_count > 0 && n >= c->E_first && n < c->E_first + c->E_count) {
            En = c->Estage + (long long)(n - c->E_first) * step;
            if (c->e_chunk_steps > 0 && !graphs) {   // host excitation still arriving:
                const int j = (n - c->E_first) / c->e_chunk_steps;   // wait for its chunk
                if (j != waited_chunk) {
                    MOT_CUDA_TRY(cudaStreamWaitEvent(s, c->e_chunk[j], 0));
                    waited_chunk = j;
                }
            }
        }
        cudaEvent_t* ev = c->profiling ? &c->events[6 * (size_t)i] : nullptr;
        if (ev) MOT_CUDA_TRY(cudaEventRecord(ev[0], s));
        history_for(c, n, s, ev ? ev + 1 : nullptr);
        if (ev) MOT_CUDA_TRY(cudaEventRecord(ev[4], s));
        mot::solve_step(c, n, En, c->norms + i, s);
        c->stats.launches += 2;
        if (ev) MOT_CUDA_TRY(cudaEventRecord(ev[5], s));
        if (J_out) {
            double* dst = J_out + (long long)i * 3 * c->M;
            if (dev_out) {
                mot::write_aos(c, n, dst, s);
            } else {
                // AoS copy into ring slot k on s, device-to-host copy on the copy
                // stream, overlapped with the next steps; slot k is rewritten only
                // after its previous copy has finished
                const int k = i % kOutSlots;
                double* slot = c->outbuf + (long long)k * step;
                MOT_CUDA_TRY(cudaStreamWaitEvent(s, c->out_done[k], 0));
                mot::write_aos(c, n, slot, s);
                MOT_CUDA_TRY(cudaEventRecord(c->out_ready[k], s));
                MOT_CUDA_TRY(cudaStreamWaitEvent(c->cstream, c->out_ready[k], 0));
                MOT_CUDA_TRY(cudaMemcpyAsync(dst, slot, sizeof(double) * step,
                                             cudaMemcpyDeviceToHost, c->cstream));
                MOT_CUDA_TRY(cudaEventRecord(c->out_done[k], c->cstream));
            }
            c->stats.launches += 1;
        }
    }

    void launch_all() {
        for (int i = 0; i < n_steps;) {
            const int n = c->n_done + 1 + i, Q = c->graph_steps;
            // a period starts where every level fires ((n - 1) mod Q = 0, Q a multiple
            // of the longest level), after step 1 (no history transform at n = 1), so all
            // periods launch the same kernels in the same order with other arguments
            if (graphs && n >= 2 && (n - 1) % Q == 0 && n_steps - i >= Q) {
                march_period_graph(c, s, [&] { for (int j = 0; j < Q; ++j) launch_step(i + j); });
                i += Q;
            } else {
                launch_step(i);
                ++i;
            }
        }
    }

    void fetch() {
        std::vector<double> nrm(n_steps);
        int hs[4];
        MOT_CUDA_TRY(cudaMemcpyAsync(nrm.data(), c->norms, sizeof(double) * n_steps,
                                     cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaMemcpyAsync(hs, c->dstatus, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
        if (J_out && !dev_out) MOT_CUDA_TRY(cudaStreamSynchronize(c->cstream));
        const int n0 = c->n_done;
        c->n_done += n_steps;
        c->last_iters = hs[0];
        c->stats.steps += n_steps;
        c->stats.cg_iters += hs[3];
        if (c->profiling) {
            for (int i = 0; i < n_steps; ++i) {
                float t[5];
                cudaEvent_t* ev = &c->events[6 * (size_t)i];
                for (int k = 0; k < 5; ++k) MOT_CUDA_TRY(cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]));
                c->stats.ms_fft_fwd += t[0];
                c->stats.ms_far += t[1];
                c->stats.ms_mac += t[2];
                c->stats.ms_fft_inv += t[3];
                c->stats.ms_solve += t[4];
            }
        }
        for (int i = 0; i < n_steps; ++i) {
            const double v = std::sqrt(nrm[i]);
            const bool bad = !std::isfinite(v) ||
                             (c->peak_norm > 0.0 && v > c->growth * c->peak_norm);
            if (bad && result == MOT_OK) {
                result = MOT_ERR_UNSTABLE;
                if (!c->fail_step) c->fail_step = n0 + 1 + i;
                char b[160];
                snprintf(b, sizeof b, "unstable: ||J_%d|| = %g (peak so far %g)", n0 + 1 + i, v,
                         c->peak_norm);
                c->err = b;
            }
            if (std::isfinite(v)) c->peak_norm = std::max(c->peak_norm, v);
            c->last_norm = v;
        }
        if (hs[1] & 4) {   // a grid barrier of the solve timed out: J from that step on is void
            result = MOT_ERR_TIMEOUT;
            c->fail_step = hs[2];
            c->broken = true;
            char b[160];
            snprintf(b, sizeof b, "timeout: a grid barrier of the solve at step %d waited longer "
                     "than %.1f s", hs[2], mot::kBarrierBudgetS);
            c->err = b;
        }
        if (result == MOT_OK && (hs[1] & 2)) {   // non-finite solve (the norm check above
            result = MOT_ERR_UNSTABLE;             // catches it too; kept for clarity)
            if (!c->fail_step) c->fail_step = hs[2];
            char b[160];
            snprintf(b, sizeof b, "unstable: NaN or Inf in the solve of step %d", hs[2]);
            c->err = b;
        }
        if (result == MOT_OK && (hs[1] & 1)) {
            result = MOT_ERR_NOT_CONVERGED;
            if (!c->fail_step) c->fail_step = hs[2];
            char b[160];
            snprintf(b, sizeof b, "CG did not converge within %d iterations at step %d",
                     c->max_iter, hs[2]);
            c->err = b;
        }
    }
};

}  // namespace

extern "C" {

mot_status mot_march(mot_ctx* c, int n_steps, double* J_out, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (c->adj_total) { c->err = "an adjoint run is open (mot_adjoint_end first)"; return MOT_ERR_ARG; }
    if (n_steps < 1) { c->err = "n_steps must be >= 1"; return MOT_ERR_ARG; }
    MarchRun run{c, n_steps, J_out, stream ? (cudaStream_t)stream : c->stream};
    mot_status st = guarded(c, [&] {
        run.begin();
        run.launch_all();
        run.fetch();
    });
    return st != MOT_OK ? st : run.result;
}

mot_status mot_eval_history(mot_ctx* c, int n_hist, const double* J_hist, double* P_out,
                            void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (c->adj_total) { c->err = "an adjoint run is open (mot_adjoint_end first)"; return MOT_ERR_ARG; }
    if (n_hist < 1 || n_hist > c->ell || !J_hist || !P_out) {
        c->err = "n_hist must be in 1..ell and buffers non-null";
        return MOT_ERR_ARG;
    }
    return guarded(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        reset_state(c, s);
        const long long step = 3 * c->M;
        double* tmp = nullptr;
        MOT_CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * step * (n_hist + 1)));
        try {
            MOT_CUDA_TRY(cudaMemcpyAsync(tmp, J_hist, sizeof(double) * step * n_hist,
                                         is_device_ptr(J_hist) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyHostToDevice, s));
            const int n = n_hist + 1;
            // J_{n-k} = J_hist[k-1]; march the rings forward through times 1..n_hist
            for (int t = 1; t <= n_hist; ++t) {
                mot::read_aos(c, tmp + (long long)(n - 1 - t) * step,
                              c->J + mot::slot_index(t, c->jring) * step, s);
                if (t < n_hist) history_for(c, t + 1, s);   // FFT of J_t into the ring
            }
            history_for(c, n, s);
            mot::history_out(c, n, tmp + (long long)n_hist * step, s);
            MOT_CUDA_TRY(cudaMemcpyAsync(P_out, tmp + (long long)n_hist * step, sizeof(double) * step,
                                         is_device_ptr(P_out) ? cudaMemcpyDeviceToDevice
                                                              : cudaMemcpyDeviceToHost, s));
            MOT_CUDA_TRY(cudaStreamSynchronize(s));
        } catch (...) {
            cudaFree(tmp);
            throw;
        }
        cudaFree(tmp);
        reset_state(c, s);
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

namespace {

// stage `count` steps of an AoS host or device array on the device (owned copy if host)
const double* on_device(mot_ctx* c, const double* src, long long count,
                        std::vector<void*>& owned, cudaStream_t s) {
    if (is_device_ptr(src)) return src;
    double* d = nullptr;
    const long long bytes = sizeof(double) * 3 * c->M * count;
    MOT_CUDA_TRY(cudaMalloc(&d, bytes));
    owned.push_back(d);
    MOT_CUDA_TRY(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
    return d;
}

void adjoint_release(mot_ctx* c) {
    cudaFree(c->adj_gchi);
    c->adj_gchi = nullptr;
    c->adj_total = 0;
    c->adj_done = 0;
    c->adjoint = false;
}

}  // namespace

mot_status mot_restart(mot_ctx* c, int n0, int n_hist, const double* J_hist, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (c->adj_total) { c->err = "an adjoint run is open (mot_adjoint_end first)"; return MOT_ERR_ARG; }
    if (n0 < 0 || n_hist < std::min(n0, c->ell) || n_hist > n0 || (n_hist > 0 && !J_hist)) {
        c->err = "mot_restart needs min(n0, ell) <= n_hist <= n0 currents J_{n0-n_hist+1..n0}";
        return MOT_ERR_ARG;
    }
    std::vector<void*> owned;
    mot_status st = guarded(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        reset_state(c, s);
        const double* Jd = n_hist ? on_device(c, J_hist, n_hist, owned, s) : nullptr;
        const long long step = 3 * c->M;
        // replay the history path over the window: every far-level firing that
        // contributes to a time after n0 happens inside it, and currents older than ell
        // steps contribute to no later time
        const int t0 = n0 - n_hist + 1;
        for (int t = t0; t <= n0; ++t) {
            mot::read_aos(c, Jd + (long long)(t - t0) * step,
                          c->J + mot::slot_index(t, c->jring) * step, s);
            if (t < n0) history_for(c, t + 1, s);
        }
        c->n_done = n0;
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
    });
    for (void* p : owned) cudaFree(p);
    return st;
}

mot_status mot_adjoint_begin(mot_ctx* c, int n_total, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (n_total < 1) { c->err = "n_total must be >= 1"; return MOT_ERR_ARG; }
    if (c->adj_total) { c->err = "an adjoint run is already open"; return MOT_ERR_ARG; }
    const mot_status st = guarded(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        MOT_CUDA_TRY(cudaMalloc(&c->adj_gchi, sizeof(double) * c->M));
        MOT_CUDA_TRY(cudaMemsetAsync(c->adj_gchi, 0, sizeof(double) * c->M, s));
        reset_state(c, s);
        c->adjoint = true;
        c->adj_total = n_total;
        c->adj_done = 0;
        MOT_CUDA_TRY(cudaMemsetAsync(c->dstatus, 0, sizeof(int) * mot::kStatusWords, s));
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
    });
    if (st != MOT_OK) adjoint_release(c);
    return st;
}

mot_status mot_adjoint_run(mot_ctx* c, int n_count, const double* J_win, int win_first,
                           int win_count, const double* dO_dJ, double* lambda, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (!c->adj_total) { c->err = "no adjoint run open (mot_adjoint_begin first)"; return MOT_ERR_ARG; }
    const int n_hi = c->adj_total - c->adj_done, n_lo = n_hi - n_count + 1;
    const int L = std::max(c->n_taps, 2);
    if (n_count < 1 || n_lo < 1 || !J_win || !dO_dJ ||
        win_first > std::max(1, n_lo - L + 1) || win_first + win_count - 1 < n_hi) {
        c->err = "adjoint run: need 1 <= n_count <= steps left and currents covering steps "
                 "max(1, n_lo - L + 1) .. n_hi (L = max(taps, 2))";
        return MOT_ERR_ARG;
    }
    mot_status result = MOT_OK;
    std::vector<void*> owned;
    mot_status st = guarded(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        const long long step = 3 * c->M;
        const double* Jd = on_device(c, J_win, win_count, owned, s);
        const double* gd = on_device(c, dO_dJ, n_count, owned, s);
        double* lamd = nullptr;
        if (lambda) {
            if (is_device_ptr(lambda)) {
                lamd = lambda;
            } else {
                MOT_CUDA_TRY(cudaMalloc(&lamd, sizeof(double) * step * n_count));
                owned.push_back(lamd);
            }
        }
        if (n_count > c->norms_cap) {
            MOT_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(c->norms);
            c->norms = nullptr;
            c->norms_cap = 0;
            MOT_CUDA_TRY(cudaMalloc(&c->norms, sizeof(double) * n_count));
            c->norms_cap = n_count;
        }
        for (int i = 0; i < n_count; ++i) {
            const int tau = c->adj_done + 1 + i;
            const int n = c->adj_total + 1 - tau;
            history_for(c, tau, s);
            mot::adjoint_step(c, tau, n, gd + (long long)(n - n_lo) * step, Jd, win_first,
                              c->adj_gchi, lamd ? lamd + (long long)(n - n_lo) * step : nullptr,
                              c->norms + i, s);
        }
        int hs[4];
        MOT_CUDA_TRY(cudaMemcpyAsync(hs, c->dstatus, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
        if (lambda && lamd != lambda)
            MOT_CUDA_TRY(cudaMemcpyAsync(lambda, lamd, sizeof(double) * step * n_count,
                                         cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
        c->adj_done += n_count;
        if (hs[1] & 4) {
            result = MOT_ERR_TIMEOUT;
            c->broken = true;
            c->err = "adjoint: a grid barrier of the solve timed out";
        } else if (hs[1] & 2) {
            result = MOT_ERR_UNSTABLE;
            c->err = "adjoint: NaN or Inf in lambda";
        } else if (hs[1] & 1) {
            result = MOT_ERR_NOT_CONVERGED;
            c->err = "adjoint: CG did not converge";
        }
    });
    for (void* p : owned) cudaFree(p);
    return st != MOT_OK ? st : result;
}

mot_status mot_adjoint_end(mot_ctx* c, double* grad_eps, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (!c->adj_total) { c->err = "no adjoint run open"; return MOT_ERR_ARG; }
    if (grad_eps && c->adj_done != c->adj_total) {
        c->err = "adjoint run incomplete: steps left";
        return MOT_ERR_ARG;
    }
    mot_status st = guarded(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        if (grad_eps) {
            std::vector<double> g(c->M), e(c->M);
            MOT_CUDA_TRY(cudaMemcpyAsync(g.data(), c->adj_gchi, sizeof(double) * c->M,
                                         cudaMemcpyDeviceToHost, s));
            MOT_CUDA_TRY(cudaMemcpyAsync(e.data(), c->eps, sizeof(double) * c->M,
                                         cudaMemcpyDeviceToHost, s));
            MOT_CUDA_TRY(cudaStreamSynchronize(s));
            for (long long m = 0; m < c->M; ++m) g[m] /= e[m] * e[m];   // dchi/deps = 1/eps^2
            MOT_CUDA_TRY(cudaMemcpy(grad_eps, g.data(), sizeof(double) * c->M,
                                    is_device_ptr(grad_eps) ? cudaMemcpyHostToDevice
                                                            : cudaMemcpyHostToHost));
        }
        c->adjoint = false;
        reset_state(c, s);
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
    });
    adjoint_release(c);
    return st;
}

mot_status mot_adjoint(mot_ctx* c, int n_steps, const double* J, const double* dO_dJ,
                       double* grad_eps, double* lambda, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (n_steps < 1 || !J || !dO_dJ || !grad_eps) {
        c->err = "n_steps >= 1 and J, dO_dJ, grad_eps non-null required";
        return MOT_ERR_ARG;
    }
    mot_status st = mot_adjoint_begin(c, n_steps, stream);
    if (st != MOT_OK) return st;
    const mot_status run = mot_adjoint_run(c, n_steps, J, 1, n_steps, dO_dJ, lambda, stream);
    if (run != MOT_OK && run != MOT_ERR_NOT_CONVERGED && run != MOT_ERR_UNSTABLE) {
        mot_adjoint_end(c, nullptr, stream);
        return run;
    }
    const std::string keep = c->err;
    st = mot_adjoint_end(c, grad_eps, stream);
    if (st != MOT_OK) return st;
    if (run != MOT_OK) c->err = keep;
    return run;
}

mot_status mot_get_table(mot_ctx* c, int l0, int n_lags, double* out) {
    if (!c) return MOT_ERR_ARG;
    if (l0 < 0 || n_lags < 1 || l0 + n_lags > c->ell + 1 || !out) {
        c->err = "lag range must lie in 0..ell";
        return MOT_ERR_ARG;
    }
    return guarded(c, [&] {
        const long long noff = (long long)c->U * c->V * c->W;
        std::vector<int> L0(noff);
        std::vector<double> tab(noff * 6 * mot::WIN);
        MOT_CUDA_TRY(cudaMemcpy(L0.data(), c->tab_l0, sizeof(int) * noff, cudaMemcpyDeviceToHost));
        MOT_CUDA_TRY(cudaMemcpy(tab.data(), c->tab, sizeof(double) * tab.size(),
                                cudaMemcpyDeviceToHost));
        for (int li = 0; li < n_lags; ++li)
            for (int cc = 0; cc < 6; ++cc)
                for (long long o = 0; o < noff; ++o) {
                    const int idx = l0 + li - L0[o];
                    out[((long long)li * 6 + cc) * noff + o] =
                        (idx >= 0 && idx < mot::WIN) ? tab[(o * 6 + cc) * mot::WIN + idx] : 0.0;
                }
    });
}

mot_status mot_get_spectrum(mot_ctx* c, int l, double* out) {
    if (!c) return MOT_ERR_ARG;
    if (l < 1 || l > c->ell || !out) { c->err = "lag must be in 1..ell"; return MOT_ERR_ARG; }
    return guarded(c, [&] { mot::spectrum_of_lag(c, l, out); });
}

mot_status mot_get_info(const mot_ctx* c, int* ell, int P[3], int* n_done, double* last_norm,
                        int* fail_step, int* last_cg_iters) {
    if (!c) return MOT_ERR_ARG;
    if (ell) *ell = c->ell;
    if (P) for (int a = 0; a < 3; ++a) P[a] = c->ax[a].P;
    if (n_done) *n_done = c->n_done;
    if (last_norm) *last_norm = c->last_norm;
    if (fail_step) *fail_step = c->fail_step;
    if (last_cg_iters) *last_cg_iters = c->last_iters;
    return c->broken ? MOT_ERR_STATE : MOT_OK;
}

mot_status mot_level_plan(int block, int ell, int scheme, int max_levels, int* n_levels, int* S,
                          int* lag0) {
    auto fail = [](const char* m) {
        g_create_error = m;
        return MOT_ERR_ARG;
    };
    if (!n_levels || max_levels < 0) return fail("n_levels must be non-null and max_levels >= 0");
    if (scheme != MOT_HISTORY_DIRECT && scheme != MOT_HISTORY_BLOCKED &&
        scheme != MOT_HISTORY_BLOCKED_DOUBLING)
        return fail("unknown history scheme");
    if (ell < 1) return fail("ell must be >= 1");
    *n_levels = 0;
    if (scheme == MOT_HISTORY_DIRECT) return MOT_OK;
    if (block < 2 || (block & (block - 1)) != 0)
        return fail("block must be a power of two >= 2 for the blocked scheme");
    int s[8], a[8];
    const int n = mot::level_plan(block, ell, scheme == MOT_HISTORY_BLOCKED, s, a);
    if (n < 0) return fail("blocked scheme: more than 8 levels needed; raise block");
    *n_levels = n;
    for (int k = 0; k < n && k < max_levels; ++k) {
        if (S) S[k] = s[k];
        if (lag0) lag0[k] = a[k];
    }
    return MOT_OK;
}

mot_status mot_get_levels(const mot_ctx* c, int max_levels, int* n_levels, int* S, int* lag0) {
    if (!c || max_levels < 0 || !n_levels) return MOT_ERR_ARG;
    const int n = c->scheme == MOT_HISTORY_BLOCKED ? c->nlev : 0;
    *n_levels = n;
    for (int k = 0; k < n && k < max_levels; ++k) {
        if (S) S[k] = c->lev_S[k];
        if (lag0) lag0[k] = c->lev_a[k];
    }
    return c->broken ? MOT_ERR_STATE : MOT_OK;
}

mot_status mot_set_solver(mot_ctx* c, double tol, int max_iter, double growth_limit) {
    if (!c) return MOT_ERR_ARG;
    if (!(tol > 0) || max_iter < 1 || !(growth_limit > 1)) {
        c->err = "tol > 0, max_iter >= 1 and growth_limit > 1 required";
        return MOT_ERR_ARG;
    }
    c->tol = tol;
    c->max_iter = max_iter;
    c->growth = growth_limit;
    for (mot_ctx* r : c->rhs_ctx) {   // the context's other right-hand sides alike
        r->tol = tol;
        r->max_iter = max_iter;
        r->growth = growth_limit;
    }
    return MOT_OK;
}

mot_status mot_set_excitation_rhs(mot_ctx* c, int n_rhs, int n_steps, const double* E,
                                  void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (n_rhs < 1 || n_rhs > 4096 || n_steps < 1 || !E) {
        c->err = "n_rhs in 1..4096, n_steps >= 1 and E non-null required";
        return MOT_ERR_ARG;
    }
    if (c->shared_src) {
        c->err = "right-hand sides belong to the context that owns the setup";
        return MOT_ERR_ARG;
    }
    const int have = 1 + (int)c->rhs_ctx.size();
    if (n_rhs != have) {
        bool fresh = c->n_done == 0;
        for (mot_ctx* r : c->rhs_ctx) fresh = fresh && r->n_done == 0;
        if (!fresh) {
            char b[160];
            snprintf(b, sizeof b, "the number of right-hand sides (%d) can change only before "
                     "the first step", have);
            c->err = b;
            return MOT_ERR_ARG;
        }
        while ((int)c->rhs_ctx.size() > n_rhs - 1) {
            mot_ctx* r = c->rhs_ctx.back();
            cudaDeviceSynchronize();
            free_all(r);
            delete r;
            c->rhs_ctx.pop_back();
        }
        while ((int)c->rhs_ctx.size() < n_rhs - 1) {
            mot_ctx* r = nullptr;
            const mot_status st = mot_create_shared(c, &r);
            if (st != MOT_OK) {
                c->err = g_create_error;
                return st;
            }
            r->max_iter = c->max_iter; r->tol = c->tol; r->growth = c->growth;
            r->graph_steps = c->graph_steps;
            r->rhs_owner = c;
            c->rhs_ctx.push_back(r);
        }
    }
    // every right-hand side is staged on one stream (the caller's, else this
    // context's, on which a device E was typically written), and each right-hand
    // side's own stream then waits for that staging
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const long long per = 3LL * c->M * n_steps;
    for (int k = 0; k < n_rhs; ++k) {
        mot_ctx* r = k == 0 ? c : c->rhs_ctx[k - 1];
        const mot_status st = mot_set_excitation(r, n_steps, E + k * per, s);
        if (st != MOT_OK) {
            if (r != c) c->err = r->err;
            return st;
        }
    }
    return guarded(c, [&] {
        cudaEvent_t staged = new_sync_event();
        MOT_CUDA_TRY(cudaEventRecord(staged, s));
        for (int k = 0; k < n_rhs; ++k) {
            mot_ctx* r = k == 0 ? c : c->rhs_ctx[k - 1];
            if (r->stream != s) MOT_CUDA_TRY(cudaStreamWaitEvent(r->stream, staged, 0));
        }
        cudaEventDestroy(staged);
    });
}

mot_status mot_march_rhs(mot_ctx* c, int n_steps, double* J_out, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (n_steps < 1) { c->err = "n_steps must be >= 1"; return MOT_ERR_ARG; }
    std::vector<mot_ctx*> all{c};
    for (mot_ctx* r : c->rhs_ctx) all.push_back(r);
    for (mot_ctx* r : all) {
        if (r->broken) return MOT_ERR_STATE;
        if (r->adj_total) { c->err = "an adjoint run is open (mot_adjoint_end first)"; return MOT_ERR_ARG; }
        if (r->n_done != c->n_done) { c->err = "right-hand sides out of step"; return MOT_ERR_ARG; }
    }
    const long long per = 3LL * c->M * n_steps;
    std::vector<MarchRun> runs;
    for (size_t k = 0; k < all.size(); ++k)
        runs.push_back(MarchRun{all[k], n_steps, J_out ? J_out + (long long)k * per : nullptr,
                                stream ? (cudaStream_t)stream : all[k]->stream});
    // the steps of all right-hand sides interleaved, each on its own stream
    mot_status st = guarded(c, [&] {
        for (MarchRun& r : runs) {
            r.graphs_allowed = false;
            r.begin();
        }
        for (int i = 0; i < n_steps; ++i)
            for (MarchRun& r : runs) r.launch_step(i);
    });
    if (st != MOT_OK) {   // a launch failed: the right-hand sides' states are not read
        for (mot_ctx* r : all) cudaStreamSynchronize(r->stream);
        cudaGetLastError();
        return st;
    }
    mot_status result = st;
    for (size_t k = 0; k < runs.size(); ++k) {
        const mot_status sk = guarded(all[k], [&] { runs[k].fetch(); });
        const mot_status rk = sk != MOT_OK ? sk : runs[k].result;
        if (result == MOT_OK && rk != MOT_OK) {
            result = rk;
            if (k) {
                char b[64];
                snprintf(b, sizeof b, "right-hand side %d: ", (int)k);
                c->err = b + all[k]->err;
            }
        }
    }
    return result;
}

mot_status mot_rhs_context(mot_ctx* c, int k, mot_ctx** out) {
    if (!c || !out) return MOT_ERR_ARG;
    *out = nullptr;
    if (k < 0 || k > (int)c->rhs_ctx.size()) {
        c->err = "right-hand side index out of range";
        return MOT_ERR_ARG;
    }
    *out = k == 0 ? c : c->rhs_ctx[k - 1];
    return MOT_OK;
}

mot_status mot_set_graph(mot_ctx* c, int steps_per_graph) {
    if (!c) return MOT_ERR_ARG;
    if (steps_per_graph < 0 || steps_per_graph > 65536) {
        c->err = "steps_per_graph must be in 0..65536";
        return MOT_ERR_ARG;
    }
    if (steps_per_graph > 0 && c->scheme == MOT_HISTORY_BLOCKED && c->nlev > 0 &&
        steps_per_graph % c->lev_period != 0) {
        char b[160];
        snprintf(b, sizeof b, "steps_per_graph must be a multiple of the longest level's "
                 "period %d", c->lev_period);
        c->err = b;
        return MOT_ERR_ARG;
    }
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    c->graph_steps = steps_per_graph;
    return MOT_OK;
}

mot_status mot_set_profiling(mot_ctx* c, int enable) {
    if (!c) return MOT_ERR_ARG;
    c->profiling = enable != 0;
    c->stats = mot_stats{};
    return MOT_OK;
}

mot_status mot_get_stats(const mot_ctx* c, mot_stats* out) {
    if (!c || !out) return MOT_ERR_ARG;
    *out = c->stats;
    return MOT_OK;
}

const char* mot_last_error(const mot_ctx* c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

// History evaluation P_{n-1} = sum_{l>=1} G_l * J_{n-l} in the spatial spectral domain
// (Sec. 3, Eq. PnFFTMOT: FFT each J once, sum the products over lags, one IFFT).
//
// Spectral ring: Jhat_{n'} is kept at slot n' mod hring (hring >= ell), so the
// forward FFT of each J runs once and is reused by every later step.  The per-bin
// product is a real symmetric 3x3 matrix times a complex 3-vector.  The stored kernel
// spectrum covers the octant k_i <= P_i/2; one load serves the four bins
// (ku, +-kv, +-kw), with the sign of the (a, b) component flipped for every mirrored
// axis among a, b (the component is odd in k_a and k_b).
//
// FP32-history: the spectra, rings and MAC are FP32; each lag's contribution is
// formed with FP32 FMAs and added into the running sum with an error-free two-sum,
// so the accumulation over up to ell lags adds no error beyond one rounding of the
// compensated total.
#include "mot_internal.cuh"

namespace {

constexpr int NT = 256;

template <typename R> struct Acc;
template <> struct Acc<double> {
    double2 s;
    __device__ void zero() { s = make_double2(0.0, 0.0); }
    __device__ void add(double2 v) { s.x += v.x; s.y += v.y; }
    __device__ double2 get() const { return s; }
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bp = s - a;
    const float ap = s - bp;
    e = (a - ap) + (b - bp);
}
template <> struct Acc<float> {
    float2 s, c;
    __device__ void zero() { s = make_float2(0.f, 0.f); c = make_float2(0.f, 0.f); }
    __device__ void add(float2 v) {
        float e;
        two_sum(s.x, v.x, s.x, e); c.x += e;
        two_sum(s.y, v.y, s.y, e); c.y += e;
    }
    __device__ float2 get() const { return make_float2(s.x + c.x, s.y + c.y); }
};

struct MacGeom {
    int Hu, Hv, Hw, Pv, Pw;
    long long nbins, noct;
};

// P^(kbins) = scale * sum_{l=l_lo}^{l_hi} Ghat_l(k) Jhat_{n-l}(k)  (+ add_in if given)
template <typename R>
__global__ void __launch_bounds__(NT) k_mac(const R* __restrict__ ghat,
                                            const typename CT<R>::c* __restrict__ ring, int hring,
                                            int n, int l_lo, int l_hi, MacGeom g, R scale,
                                            typename CT<R>::c* __restrict__ phat) {
    typedef typename CT<R>::c C;
    const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= g.noct) return;
    const int ku = (int)(o % g.Hu);
    const int kv = (int)((o / g.Hu) % g.Hv);
    const int kw = (int)(o / ((long long)g.Hu * g.Hv));
    const bool mv = kv > 0 && 2 * kv < g.Pv;
    const bool mw = kw > 0 && 2 * kw < g.Pw;
    long long bidx[4];
    bool valid[4];
    bidx[0] = ((long long)kw * g.Pv + kv) * g.Hu + ku;
    bidx[1] = ((long long)kw * g.Pv + (g.Pv - kv)) * g.Hu + ku;
    bidx[2] = ((long long)(g.Pw - kw) * g.Pv + kv) * g.Hu + ku;
    bidx[3] = ((long long)(g.Pw - kw) * g.Pv + (g.Pv - kv)) * g.Hu + ku;
    valid[0] = true;
    valid[1] = mv;
    valid[2] = mw;
    valid[3] = mv && mw;
    // sign of (xy, xz, yz) in each mirror
    const R sxy[4] = {(R)1, (R)-1, (R)1, (R)-1};
    const R sxz[4] = {(R)1, (R)1, (R)-1, (R)-1};
    const R syz[4] = {(R)1, (R)-1, (R)-1, (R)1};
    Acc<R> acc[4][3];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[m][a].zero();
    const long long slot_stride = 3 * g.nbins;
    for (int l = l_lo; l <= l_hi; ++l) {
        const R* gp = ghat + (long long)(l - 1) * 6 * g.noct + o;
        const R gxx = gp[0], gyy = gp[g.noct], gzz = gp[2 * g.noct];
        const R gxy = gp[3 * g.noct], gxz = gp[4 * g.noct], gyz = gp[5 * g.noct];
        const long long slot = (((long long)(n - l)) % hring + hring) % hring;
        const C* base = ring + slot * slot_stride;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (!valid[m]) continue;
            const C x = base[bidx[m]];
            const C y = base[g.nbins + bidx[m]];
            const C z = base[2 * g.nbins + bidx[m]];
            const R a = sxy[m] * gxy, b = sxz[m] * gxz, cc = syz[m] * gyz;
            C ox, oy, oz;
            ox.x = gxx * x.x + a * y.x + b * z.x;
            ox.y = gxx * x.y + a * y.y + b * z.y;
            oy.x = a * x.x + gyy * y.x + cc * z.x;
            oy.y = a * x.y + gyy * y.y + cc * z.y;
            oz.x = b * x.x + cc * y.x + gzz * z.x;
            oz.y = b * x.y + cc * y.y + gzz * z.y;
            acc[m][0].add(ox);
            acc[m][1].add(oy);
            acc[m][2].add(oz);
        }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (!valid[m]) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C v = acc[m][a].get();
            v.x *= scale;
            v.y *= scale;
            phat[a * g.nbins + bidx[m]] = v;
        }
    }
}

MacGeom geom(const mot_ctx* c) {
    MacGeom g;
    g.Hu = c->Hu; g.Hv = c->Hv; g.Hw = c->Hw;
    g.Pv = c->ax[1].P; g.Pw = c->ax[2].P;
    g.nbins = c->nbins; g.noct = c->noct;
    return g;
}

}  // namespace

namespace mot {

template <typename R>
void history_alloc(mot_ctx* c) {
    typedef typename CT<R>::c C;
    HistoryBuffers<R>& hb = hbuf<R>(c);
    c->hring = c->ell;
    const long long slot = 3 * c->nbins;
    MOT_CUDA_TRY(cudaMalloc(&hb.jhat_ring, sizeof(C) * slot * c->hring));
    MOT_CUDA_TRY(cudaMalloc(&hb.ghat, sizeof(R) * 6 * c->noct * c->ell));
    MOT_CUDA_TRY(cudaMalloc(&hb.phat, sizeof(C) * slot));
    MOT_CUDA_TRY(cudaMalloc(&hb.tmp1, sizeof(C) * 3LL * c->W * c->V * c->Hu));
    MOT_CUDA_TRY(cudaMalloc(&hb.tmp2, sizeof(C) * 3LL * c->W * c->ax[1].P * c->Hu));
    MOT_CUDA_TRY(cudaMalloc(&hb.hist_spatial, sizeof(R) * 3 * c->M));
}

template <typename R>
void history_free(mot_ctx* c) {
    HistoryBuffers<R>& hb = hbuf<R>(c);
    cudaFree(hb.jhat_ring);
    cudaFree(hb.ghat);
    cudaFree(hb.phat);
    cudaFree(hb.tmp1);
    cudaFree(hb.tmp2);
    cudaFree(hb.hist_spatial);
    cudaFree(hb.acc_ring);
    cudaFree(hb.level_spec);
    hb = HistoryBuffers<R>();
}

template <typename R>
void history_reset(mot_ctx* c, cudaStream_t s) {
    typedef typename CT<R>::c C;
    HistoryBuffers<R>& hb = hbuf<R>(c);
    MOT_CUDA_TRY(cudaMemsetAsync(hb.jhat_ring, 0, sizeof(C) * 3 * c->nbins * c->hring, s));
}

// hist_spatial <- sum_{l=1}^{ell} G_l * J_{n-l}; J_{n-1} is read from the spatial ring
template <typename R>
void history_step(mot_ctx* c, int n, cudaStream_t s, cudaEvent_t ev_fwd, cudaEvent_t ev_mac) {
    HistoryBuffers<R>& hb = hbuf<R>(c);
    const long long slot = 3 * c->nbins;
    if (n >= 2) {
        const double* Jprev = c->J + slot_index(n - 1, c->jring) * 3 * c->M;
        fft_forward<R>(c, Jprev, hb.jhat_ring + slot_index(n - 1, c->hring) * slot, s);
        c->stats.launches += 3;
    }
    if (ev_fwd) MOT_CUDA_TRY(cudaEventRecord(ev_fwd, s));
    const R scale = (R)(1.0 / ((double)c->ax[0].P * c->ax[1].P * c->ax[2].P));
    k_mac<R><<<(int)((c->noct + NT - 1) / NT), NT, 0, s>>>(hb.ghat, hb.jhat_ring, c->hring, n, 1,
                                                           c->ell, geom(c), scale, hb.phat);
    MOT_LAUNCH_CHECK();
    c->stats.launches += 1;
    c->stats.mac_launches += 1;
    if (ev_mac) MOT_CUDA_TRY(cudaEventRecord(ev_mac, s));
    fft_inverse<R>(c, hb.phat, hb.hist_spatial, s);
    c->stats.launches += 3;
}

template void history_alloc<double>(mot_ctx*);
template void history_alloc<float>(mot_ctx*);
template void history_free<double>(mot_ctx*);
template void history_free<float>(mot_ctx*);
template void history_reset<double>(mot_ctx*, cudaStream_t);
template void history_reset<float>(mot_ctx*, cudaStream_t);
template void history_step<double>(mot_ctx*, int, cudaStream_t, cudaEvent_t, cudaEvent_t);
template void history_step<float>(mot_ctx*, int, cudaStream_t, cudaEvent_t, cudaEvent_t);

}  // namespace mot

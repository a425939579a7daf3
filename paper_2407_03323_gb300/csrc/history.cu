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

// Phat(k) = scale * sum_{l=1}^{L} Ghat_l(k) Jhat_{n-l}(k) over all rfft bins.
// A warp covers 8 consecutive octant bins (ku) x 4 mirrors: lane = mirror * 8 + j.
// The 8 lanes of a mirror read 8 consecutive bins of a ring row; the kernel values of
// the 8 bins ([lag][octant bin][6], 6 per bin) are one contiguous load shared by the
// 4 mirror groups.  Ring slots are walked backwards from slot_first = (n-1) mod hring.
template <typename R>
__global__ void __launch_bounds__(NT) k_mac(const R* __restrict__ ghat,
                                            const typename CT<R>::c* __restrict__ ring, int hring,
                                            int slot_first, int L, MacGeom g, R scale,
                                            typename CT<R>::c* __restrict__ phat) {
    typedef typename CT<R>::c C;
    typedef typename std::conditional<std::is_same<R, double>::value, double2, float2>::type R2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int mirror = lane >> 3, j = lane & 7;
    const long long o = ((long long)blockIdx.x * (NT / 32) + warp) * 8 + j;
    if (o >= g.noct) return;
    const int ku = (int)(o % g.Hu);
    const int kv = (int)((o / g.Hu) % g.Hv);
    const int kw = (int)(o / ((long long)g.Hu * g.Hv));
    const bool mv = kv > 0 && 2 * kv < g.Pv;
    const bool mw = kw > 0 && 2 * kw < g.Pw;
    const bool fv = (mirror & 1) != 0, fw = (mirror & 2) != 0;
    if ((fv && !mv) || (fw && !mw)) return;
    const int kv2 = fv ? g.Pv - kv : kv;
    const int kw2 = fw ? g.Pw - kw : kw;
    const long long bidx = ((long long)kw2 * g.Pv + kv2) * g.Hu + ku;
    const R sxy = fv ? (R)-1 : (R)1;
    const R sxz = fw ? (R)-1 : (R)1;
    const R syz = (fv != fw) ? (R)-1 : (R)1;
    Acc<R> ax, ay, az;
    ax.zero(); ay.zero(); az.zero();
    const long long slot_stride = 3 * g.nbins;
    int slot = slot_first;
    const R2* gp = reinterpret_cast<const R2*>(ghat + o * 6);
    const long long gstep = g.noct * 3;   // in R2 units per lag
#pragma unroll 2
    for (int l = 1; l <= L; ++l) {
        const R2 g01 = gp[0], g23 = gp[1], g45 = gp[2];
        gp += gstep;
        const C* base = ring + (long long)slot * slot_stride + bidx;
        const C x = base[0];
        const C y = base[g.nbins];
        const C z = base[2 * g.nbins];
        slot = slot == 0 ? hring - 1 : slot - 1;
        const R gxx = g01.x, gyy = g01.y, gzz = g23.x;
        const R a = sxy * g23.y, b = sxz * g45.x, cc = syz * g45.y;
        C ox, oy, oz;
        ox.x = gxx * x.x + a * y.x + b * z.x;
        ox.y = gxx * x.y + a * y.y + b * z.y;
        oy.x = a * x.x + gyy * y.x + cc * z.x;
        oy.y = a * x.y + gyy * y.y + cc * z.y;
        oz.x = b * x.x + cc * y.x + gzz * z.x;
        oz.y = b * x.y + cc * y.y + gzz * z.y;
        ax.add(ox);
        ay.add(oy);
        az.add(oz);
    }
    C v = ax.get(); v.x *= scale; v.y *= scale; phat[bidx] = v;
    v = ay.get(); v.x *= scale; v.y *= scale; phat[g.nbins + bidx] = v;
    v = az.get(); v.x *= scale; v.y *= scale; phat[2 * g.nbins + bidx] = v;
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
    const long long nblk = (c->noct + 8 * (NT / 32) - 1) / (8 * (NT / 32));
    k_mac<R><<<(int)nblk, NT, 0, s>>>(hb.ghat, hb.jhat_ring, c->hring,
                                      (int)slot_index(n - 1, c->hring), c->ell, geom(c), scale,
                                      hb.phat);
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

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
// Blocked temporal scheme (Secs. 4-5, MOT_HISTORY_BLOCKED): lags 1..B-1 are multiplied
// every step as above; the lags [a, a + S) form a level of length S, with a = S for
// S = B, 2B, 4B, ... and, where the last of these would reach far past ell, a shorter
// last level over the remaining lags (history_alloc).  At every step n0 with
// (n0 - 1) mod S = 0 the level computes its contribution to the next S histories,
// y(n0 + j) = sum_{l=a}^{a+S-1} Ghat_l Jhat(n0 + j - l), j < S, as one block Toeplitz
// product by overlap-save: per spectral bin a length-2S FFT over time of the window
// Jhat(n0 - a - S .. n0 - a + S - 1) (read from the ring; with a >= S all of it lies
// before n0), a product with the precomputed temporal spectrum of
// [Ghat_a .. Ghat_{a+S-1}, 0 .. 0], an inverse FFT, and the last S outputs written to
// that level's own ring of future-history accumulators (S slots).
// Every time is covered by exactly one firing of each level, so a firing only stores
// (no read-modify-write), and the per-step near MAC adds every level's entry for its
// step.  A level's inputs are all older than n0,
// so the scheme is causal (the division of Sec. 4.1 into Toeplitz blocks that use only
// computed currents); levels double in length so a step costs O(log ell) block work on
// average, the temporal counterpart of Eq. ComplexityHierarchicalDivisionInTime.
#include "mot_internal.cuh"
#include "fft_core.cuh"

#include <algorithm>

using namespace mot_fft;

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

// this step's entries of the far levels' accumulator rings ([3][nbins] each)
template <typename C> struct FarSums {
    const C* p[8];
    int n;
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
                                            typename CT<R>::c* __restrict__ phat,
                                            FarSums<typename CT<R>::c> far) {
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
    for (int k = 0; k < far.n; ++k) {   // far-lag contributions of this step
        const C* f = far.p[k];
        ax.add(f[bidx]);
        ay.add(f[g.nbins + bidx]);
        az.add(f[2 * g.nbins + bidx]);
    }
    const long long slot_stride = 3 * g.nbins;
    int slot = slot_first;
    const R2* gp = reinterpret_cast<const R2*>(ghat + o * 6);
    const long long gstep = g.noct * 3;   // in R2 units per lag
#pragma unroll 8
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

// temporal spectra of the level of length S over lags [a, a + S):
// H(w) = sum_{m=0}^{lmax-a} Ghat_{a+m} exp(-2 pi i w m / (2S)), lmax = min(a + S - 1, ell),
// w = 0..S (the rest follows by H(2S - w) = conj H(w)); out [w][6][octant bin], one
// plane per component so that a warp over consecutive bins reads one contiguous run
template <typename R>
__global__ void k_level_spec(const R* __restrict__ ghat, long long noct, int S, int a, int lmax,
                             const double2* __restrict__ tw, typename CT<R>::c* __restrict__ out) {
    typedef typename CT<R>::c C;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= noct * (S + 1)) return;
    const long long o = i % noct;
    const int w = (int)(i / noct);
    double2 acc[6];
    for (int c = 0; c < 6; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int m = 0; m <= lmax - a; ++m) {
        const double2 t = tw[((long long)w * m) % (2 * S)];
        const R* gp = ghat + ((long long)(a + m - 1) * noct + o) * 6;
        for (int c = 0; c < 6; ++c) {
            const double g = (double)gp[c];
            acc[c].x += g * t.x;
            acc[c].y += g * t.y;
        }
    }
    C* op = out + (long long)w * 6 * noct + o;
    for (int c = 0; c < 6; ++c) {
        C v;
        v.x = acc[c].x;
        v.y = acc[c].y;
        op[c * noct] = v;
    }
}

constexpr int kMaxLevel = 256;   // longest level S (window 2S in shared memory)

template <typename R> struct FarArgs {
    typedef typename CT<R>::c C;
    const C* ring;
    int hring;
    long long nbins, noct;
    const C* H;          // level spectra [S+1][6][noct]
    C* acc;              // this level's accumulator ring [smax][3][nbins]
    int smax;            // its length (S)
    int n0, S, lmax;
    int w0;              // window start n0 - a - S (a the level's first lag): time of x[0]
    int Hu, Hv, Hw, Pv, Pw;
    int ntile;
    RadixList rl;        // length 2S
    const C* tw;
};

// one level firing at step n0: writes y(n0 + j), j < S, to the level's accumulator ring
template <typename R, int TB>
__global__ void __launch_bounds__(NT) k_far(FarArgs<R> a) {
    typedef typename CT<R>::c C;
    constexpr int L3 = 3 * TB;
    constexpr int ld = L3 + 1;
    const int P = 2 * a.S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* stw = reinterpret_cast<C*>(smem_raw);
    C* b0 = stw + tw_entries<C>(P);
    C* b1 = b0 + P * ld;
    // block -> (octant row, mirror, ku tile); the four mirrors of a row are adjacent
    const int ut = blockIdx.x % a.ntile;
    const int rest = blockIdx.x / a.ntile;
    const int mirror = rest & 3;
    const int orow = rest >> 2;
    const int kv_o = orow % a.Hv, kw_o = orow / a.Hv;
    const bool fv = (mirror & 1) != 0, fw = (mirror & 2) != 0;
    const bool mv = kv_o > 0 && 2 * kv_o < a.Pv;
    const bool mw = kw_o > 0 && 2 * kw_o < a.Pw;
    if ((fv && !mv) || (fw && !mw)) return;
    const int kv = fv ? a.Pv - kv_o : kv_o;
    const int kw = fw ? a.Pw - kw_o : kw_o;
    const int ku0 = ut * TB;
    const long long row = ((long long)kw * a.Pv + kv) * a.Hu + ku0;
    const long long orow_base = ((long long)kw_o * a.Hv + kv_o) * a.Hu + ku0;
    const R sxy = fv ? (R)-1 : (R)1;
    const R sxz = fw ? (R)-1 : (R)1;
    const R syz = (fv != fw) ? (R)-1 : (R)1;
    // ring slot of every window time (-1: older than the level's lags or before t = 1)
    // and accumulator slot of every output time
    __shared__ int s_in[2 * kMaxLevel];
    __shared__ int s_out[kMaxLevel];
    const int tfirst = max(1, a.n0 - a.lmax);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int time = a.w0 + i;
        s_in[i] = time >= tfirst ? time % a.hring : -1;
        if (i < a.S) s_out[i] = (a.n0 + i) % a.smax;
    }
    load_tw(stw, a.tw, P);
    __syncthreads();
    for (int it = threadIdx.x; it < P * L3; it += blockDim.x) {
        const int i = it / L3, t = it % L3;
        const int comp = t / TB, bb = t % TB;
        const int slot = s_in[i];
        const bool ok = slot >= 0 && ku0 + bb < a.Hu;
        cp_async_c(&b0[i * ld + t],
                   ok ? a.ring + ((long long)slot * 3 + comp) * a.nbins + row + bb : a.ring, ok);
    }
    cp_async_commit_wait();
    __syncthreads();
    C* X = fft_tile<C, L3>(b0, b1, P, a.rl.r, a.rl.n, ld, stw, -1);
    C* other = (X == b0) ? b1 : b0;
    for (int it = threadIdx.x; it < P * TB; it += blockDim.x) {
        const int w = it / TB, bb = it % TB;
        if (ku0 + bb >= a.Hu) continue;
        const bool cj = w > a.S;
        const int ws = cj ? P - w : w;
        const C* hp = a.H + (long long)ws * 6 * a.noct + orow_base + bb;
        C h[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            h[c] = hp[c * a.noct];
            if (cj) h[c].y = -h[c].y;
        }
        h[3].x *= sxy; h[3].y *= sxy;
        h[4].x *= sxz; h[4].y *= sxz;
        h[5].x *= syz; h[5].y *= syz;
        C* xp = X + w * ld + bb;
        const C x0 = xp[0], x1 = xp[TB], x2 = xp[2 * TB];
        xp[0] = cadd(cadd(cmul(h[0], x0), cmul(h[3], x1)), cmul(h[4], x2));
        xp[TB] = cadd(cadd(cmul(h[3], x0), cmul(h[1], x1)), cmul(h[5], x2));
        xp[2 * TB] = cadd(cadd(cmul(h[4], x0), cmul(h[5], x1)), cmul(h[2], x2));
    }
    __syncthreads();
    C* Y = fft_tile<C, L3>(X, other, P, a.rl.r, a.rl.n, ld, stw, +1);
    const R scale = (R)1 / (R)P;
    for (int it = threadIdx.x; it < a.S * L3; it += blockDim.x) {
        const int j = it / L3, t = it % L3;
        const int comp = t / TB, bb = t % TB;
        if (ku0 + bb >= a.Hu) continue;
        const long long slot = s_out[j];
        C* dst = a.acc + (slot * 3 + comp) * a.nbins + row + bb;
        const C y = Y[(a.S + j) * ld + t];
        C v;
        v.x = y.x * scale;
        v.y = y.y * scale;
        *dst = v;
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

// doubling levels: lags [S, 2S) for S = B, 2B, ... while S <= ell.  The last of them may
// reach far beyond ell (at 104^3, ell = 182: [128, 256) for 55 live lags).  With fit,
// when the lags left for it, [a, ell], number at most a / 2, it becomes the shortest
// level S' = B 2^j >= ell - a + 1 over [a, a + S'): a Toeplitz block needs only S' <= a
// to use computed currents alone, and a level costs per step about the same bytes
// whatever S but fewer butterflies for a shorter transform (the 2S = 256 transform of
// the example fires for 55 lags)
int level_plan(int block, int ell, bool fit, int S[8], int a[8]) {
    int n = 0;
    for (long long s = block; s <= ell; s *= 2) {
        if (n == 8) return -1;
        S[n] = (int)s;
        a[n] = (int)s;
        ++n;
    }
    if (fit && n >= 2) {
        const int rest = ell - a[n - 1] + 1;
        int s = block;
        while (s < rest) s *= 2;
        if (s < S[n - 1]) S[n - 1] = s;
    }
    return n;
}

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
    if (c->scheme == MOT_HISTORY_BLOCKED) {
        const int nl = level_plan(c->block, c->ell, c->lev_fit, c->lev_S, c->lev_a);
        if (nl < 0)
            throw MotError{MOT_ERR_ARG, "blocked scheme: more than 8 levels needed; raise block"};
        c->nlev = nl;
        long long spec = 0;
        c->lev_period = 1;
        for (int k = 0; k < c->nlev; ++k) {
            const int S = c->lev_S[k];
            c->lev_off[k] = spec;
            spec += (long long)(S + 1) * c->noct * 6;
            fft_plan_axis(c->lev_fft[k], 2 * S);
            c->lev_period = std::max(c->lev_period, S);
        }
        // one accumulator ring per level (S slots each): every firing writes its
        // outputs, the near MAC of a step sums the levels' entries for that step
        long long acc_slots = 0;
        for (int k = 0; k < c->nlev; ++k) {
            c->lev_acc[k] = acc_slots;
            acc_slots += c->lev_S[k];
        }
        c->smax = std::max<long long>(acc_slots, 1);
        MOT_CUDA_TRY(cudaMalloc(&hb.level_spec, sizeof(C) * std::max<long long>(spec, 1)));
        MOT_CUDA_TRY(cudaMalloc(&hb.acc_ring, sizeof(C) * slot * c->smax));
    }
}

// march-state buffers of a context that shares src's kernel and level spectra
template <typename R>
void history_alloc_shared(mot_ctx* c, mot_ctx* src) {
    typedef typename CT<R>::c C;
    HistoryBuffers<R>& hb = hbuf<R>(c);
    const HistoryBuffers<R>& sb = hbuf<R>(src);
    const long long slot = 3 * c->nbins;
    hb.ghat = sb.ghat;
    hb.level_spec = sb.level_spec;
    MOT_CUDA_TRY(cudaMalloc(&hb.jhat_ring, sizeof(C) * slot * c->hring));
    MOT_CUDA_TRY(cudaMalloc(&hb.phat, sizeof(C) * slot));
    MOT_CUDA_TRY(cudaMalloc(&hb.tmp1, sizeof(C) * 3LL * c->W * c->V * c->Hu));
    MOT_CUDA_TRY(cudaMalloc(&hb.tmp2, sizeof(C) * 3LL * c->W * c->ax[1].P * c->Hu));
    MOT_CUDA_TRY(cudaMalloc(&hb.hist_spatial, sizeof(R) * 3 * c->M));
    if (c->scheme == MOT_HISTORY_BLOCKED)
        MOT_CUDA_TRY(cudaMalloc(&hb.acc_ring, sizeof(C) * slot * c->smax));
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
    if (hb.acc_ring)
        MOT_CUDA_TRY(cudaMemsetAsync(hb.acc_ring, 0, sizeof(C) * 3 * c->nbins * c->smax, s));
}

// temporal spectra of every level from the spatial spectra (setup)
template <typename R>
void level_spectra(mot_ctx* c) {
    HistoryBuffers<R>& hb = hbuf<R>(c);
    for (int k = 0; k < c->nlev; ++k) {
        const int S = c->lev_S[k], a = c->lev_a[k];
        const int lmax = std::min(a + S - 1, c->ell);
        const long long n = c->noct * (S + 1);
        k_level_spec<R><<<(int)((n + NT - 1) / NT), NT, 0, c->stream>>>(
            hb.ghat, c->noct, S, a, lmax, c->lev_fft[k].tw64, hb.level_spec + c->lev_off[k]);
        MOT_LAUNCH_CHECK();
    }
    MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
}

template <typename R> const typename CT<R>::c* twtab(const AxisFFT& a);
template <> const double2* twtab<double>(const AxisFFT& a) { return a.tw64; }
template <> const float2* twtab<float>(const AxisFFT& a) { return a.tw32; }

// ---------------------------------------------------------------- register variant
// For 2S <= 64: one thread per (bin, component) line.  A block is three warps (warp =
// component) over 32 consecutive bins of one rfft row.  Each thread loads its 2S window
// samples (coalesced across the warp), runs an unrolled radix-2 DIF FFT in registers
// (output in bit-reversed order), the three spectra are exchanged through shared memory
// for the 3x3 product (frequency of slot i is bitrev(i)), and an unrolled radix-2 DIT
// inverse (bit-reversed input, natural output) leaves the block outputs in registers.
template <int P> __host__ __device__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1, k = P >> 1; b < P; b <<= 1, k >>= 1)
        if (i & b) r |= k;
    return r;
}

// compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1
template <int B, int E> struct Unroll {
    template <typename F> __device__ __forceinline__ static void run(F&& f) {
        f(std::integral_constant<int, B>());
        Unroll<B + 1, E>::run(f);
    }
};
template <int E> struct Unroll<E, E> {
    template <typename F> __device__ __forceinline__ static void run(F&&) {}
};

// Lines of length P = T * Q are split over T threads; thread t holds positions
// t Q .. t Q + Q - 1 of the (natural- or bit-reversed-order) line.  Stages whose span
// reaches across threads exchange values with the partner thread by warp shuffles
// (lane = t * (32 / T) + line) and take their twiddles from a shared table of the P
// roots; the others are register-local with literal twiddles.

// local DIF stage of span LEN (<= Q) over the thread's Q values
template <typename C, int Q, int LEN, int DIR>
__device__ __forceinline__ void dif_local(C* x) {
    constexpr int half = LEN / 2;
    Unroll<0, Q / 2>::run([&](auto q) {
        constexpr int st = (decltype(q)::value / half) * LEN;
        constexpr int k = decltype(q)::value % half;
        const C a = x[st + k], b = x[st + k + half];
        x[st + k] = cadd(a, b);
        x[st + k + half] = twiddle_c<k, LEN, DIR>(csub(a, b));
    });
}

template <typename C, int Q, int LEN, int DIR>
__device__ __forceinline__ void dit_local(C* x) {
    constexpr int half = LEN / 2;
    Unroll<0, Q / 2>::run([&](auto q) {
        constexpr int st = (decltype(q)::value / half) * LEN;
        constexpr int k = decltype(q)::value % half;
        const C a = x[st + k];
        const C b = twiddle_c<k, LEN, DIR>(x[st + k + half]);
        x[st + k] = cadd(a, b);
        x[st + k + half] = csub(a, b);
    });
}

__device__ __forceinline__ float2 shfl_c(float2 v, int mask) {
    v.x = __shfl_xor_sync(0xffffffffu, v.x, mask);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, mask);
    return v;
}
__device__ __forceinline__ double2 shfl_c(double2 v, int mask) {
    v.x = __shfl_xor_sync(0xffffffffu, v.x, mask);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, mask);
    return v;
}

// cross-thread DIF stage: span LEN = 2 * HT * Q, partner thread t ^ HT
template <typename C, int Q, int T, int HT, int DIR>
__device__ __forceinline__ void dif_cross(C* x, const C* __restrict__ tw, int t) {
    constexpr int P = Q * T, LEN = 2 * HT * Q, ts = P / LEN;
    const bool upper = (t & HT) == 0;
    const int base = ((t & ~HT) * Q) % LEN;
    Unroll<0, Q>::run([&](auto q) {
        constexpr int j = decltype(q)::value;
        const C mine = x[j];
        const C other = shfl_c(mine, HT * (32 / T));
        if (upper) x[j] = cadd(mine, other);
        else x[j] = twmul_tab(tw, (base + j) * ts, P, DIR, csub(other, mine));
    });
}

template <typename C, int Q, int T, int HT, int DIR>
__device__ __forceinline__ void dit_cross(C* x, const C* __restrict__ tw, int t) {
    constexpr int P = Q * T, LEN = 2 * HT * Q, ts = P / LEN;
    const bool upper = (t & HT) == 0;
    const int base = ((t & ~HT) * Q) % LEN;
    Unroll<0, Q>::run([&](auto q) {
        constexpr int j = decltype(q)::value;
        C send = x[j];
        if (!upper) send = twmul_tab(tw, (base + j) * ts, P, DIR, send);
        const C recv = shfl_c(send, HT * (32 / T));
        x[j] = upper ? cadd(send, recv) : csub(recv, send);
    });
}

template <typename C, int Q, int T, int LEN, int DIR> struct DifLoc {
    __device__ __forceinline__ static void run(C* x) {
        dif_local<C, Q, LEN, DIR>(x);
        DifLoc<C, Q, T, LEN / 2, DIR>::run(x);
    }
};
template <typename C, int Q, int T, int DIR> struct DifLoc<C, Q, T, 1, DIR> {
    __device__ __forceinline__ static void run(C*) {}
};
template <typename C, int Q, int T, int LEN, int DIR> struct DitLoc {
    __device__ __forceinline__ static void run(C* x) {
        dit_local<C, Q, LEN, DIR>(x);
        DitLoc<C, Q, T, LEN * 2, DIR>::run(x);
    }
};
template <typename C, int Q, int T, int DIR> struct DitLoc<C, Q, T, 2 * Q, DIR> {
    __device__ __forceinline__ static void run(C*) {}
};
template <typename C, int Q, int T, int HT, int DIR> struct DifCross {
    __device__ __forceinline__ static void run(C* x, const C* tw, int t) {
        dif_cross<C, Q, T, HT, DIR>(x, tw, t);
        DifCross<C, Q, T, HT / 2, DIR>::run(x, tw, t);
    }
};
template <typename C, int Q, int T, int DIR> struct DifCross<C, Q, T, 0, DIR> {
    __device__ __forceinline__ static void run(C*, const C*, int) {}
};
template <typename C, int Q, int T, int HT, int DIR> struct DitCross {
    __device__ __forceinline__ static void run(C* x, const C* tw, int t) {
        dit_cross<C, Q, T, HT, DIR>(x, tw, t);
        DitCross<C, Q, T, HT * 2, DIR>::run(x, tw, t);
    }
};
template <typename C, int Q, int T, int DIR> struct DitCross<C, Q, T, T, DIR> {
    __device__ __forceinline__ static void run(C*, const C*, int) {}
};

// natural order in, bit-reversed out: cross stages (span > Q) first, then local
template <typename C, int Q, int T, int DIR>
__device__ __forceinline__ void fft_dif_reg(C* x, const C* __restrict__ tw, int t) {
    DifCross<C, Q, T, T / 2, DIR>::run(x, tw, t);
    DifLoc<C, Q, T, Q, DIR>::run(x);
}
// bit-reversed in, natural order out: local stages first, then cross
template <typename C, int Q, int T, int DIR>
__device__ __forceinline__ void fft_dit_reg(C* x, const C* __restrict__ tw, int t) {
    DitLoc<C, Q, T, 2, DIR>::run(x);
    DitCross<C, Q, T, 1, DIR>::run(x, tw, t);
}

template <typename R, int Q, int T> struct FarRegSmem {
    typedef typename CT<R>::c C;
    static constexpr int P = Q * T, S = P / 2, NB = 32 / T;
    C X[P][3][NB];          // forward spectra of the three components
    C H[S + 1][6][NB];      // the block's level spectra, w = 0..S
    C tw[tw_entries<C>(P)]; // roots of unity for the cross-thread stages (FP32: hi, lo)
    int in[P];              // ring slot of every window time (-1: none)
    int out[S];             // accumulator slot of every output time
};

// One level firing at step n0: y(n0 + j), j < S, written to the level's accumulator
// ring.  Block = three warps (warp = component) over 32 / T bins of one rfft row.
// The block's kernel spectra are copied to shared memory asynchronously while the
// window is loaded and transformed.  Mirror signs: the off-diagonal spectra of the
// mirrored rows flip as s_ab = sigma_a sigma_b (sigma_x = 1, sigma_y = -1 if v is
// mirrored, sigma_z = -1 if w is), so the product uses the octant spectra on
// sigma-scaled inputs and scales each output row by its sigma.
template <typename R, int Q, int T>
__global__ void __launch_bounds__(96) k_far_reg(FarArgs<R> a) {
    typedef typename CT<R>::c C;
    typedef FarRegSmem<R, Q, T> SM;
    constexpr int P = SM::P, S = SM::S, NB = SM::NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    const int comp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = lane / NB, line = lane % NB;
    const int ut = blockIdx.x % a.ntile;
    const int rest = blockIdx.x / a.ntile;
    const int mirror = rest & 3;
    const int orow = rest >> 2;
    const int kv_o = orow % a.Hv, kw_o = orow / a.Hv;
    const bool fv = (mirror & 1) != 0, fw = (mirror & 2) != 0;
    const bool mv = kv_o > 0 && 2 * kv_o < a.Pv;
    const bool mw = kw_o > 0 && 2 * kw_o < a.Pw;
    if ((fv && !mv) || (fw && !mw)) return;
    const int kv = fv ? a.Pv - kv_o : kv_o;
    const int kw = fw ? a.Pw - kw_o : kw_o;
    const int ku0 = ut * NB;
    const int nlive = min(NB, a.Hu - ku0);
    const bool live = line < nlive;
    const long long row = ((long long)kw * a.Pv + kv) * a.Hu + ku0 + line;
    const long long obase = ((long long)kw_o * a.Hv + kv_o) * a.Hu + ku0;
    for (int i = threadIdx.x; i < (S + 1) * 6 * NB; i += blockDim.x) {
        const int l = i % NB;
        if (l < nlive) cp_async_c(&sm.H[0][0][0] + i, a.H + (long long)(i / NB) * a.noct + obase + l);
    }
    const int tfirst = max(1, a.n0 - a.lmax);
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int time = a.w0 + i;
        sm.in[i] = time >= tfirst ? time % a.hring : -1;
        if (i < S) sm.out[i] = (a.n0 + i) % a.smax;
    }
    for (int i = threadIdx.x; i < tw_entries<C>(P); i += blockDim.x) sm.tw[i] = a.tw[i];
    __syncthreads();
    const R sig = comp == 0 ? (R)1 : (comp == 1 ? (fv ? (R)-1 : (R)1) : (fw ? (R)-1 : (R)1));
    C x[Q];
    Unroll<0, Q>::run([&](auto q) {
        constexpr int j = decltype(q)::value;
        const int slot = sm.in[t * Q + j];
        C v;
        v.x = 0; v.y = 0;
        if (slot >= 0 && live) v = a.ring[((long long)slot * 3 + comp) * a.nbins + row];
        x[j] = v;
    });
    fft_dif_reg<C, Q, T, -1>(x, sm.tw, t);
    Unroll<0, Q>::run([&](auto q) {
        constexpr int j = decltype(q)::value;
        C v = x[j];
        v.x *= sig; v.y *= sig;
        sm.X[t * Q + j][comp][line] = v;
    });
    cp_async_commit_wait();
    __syncthreads();
    // row `comp` of the symmetric 3x3: components (xx, yy, zz, xy, xz, yz) = 0..5
    const int i0 = comp == 0 ? 0 : (comp == 1 ? 3 : 4);
    const int i1 = comp == 0 ? 3 : (comp == 1 ? 1 : 5);
    const int i2 = comp == 0 ? 4 : (comp == 1 ? 5 : 2);
    const int brt = bitrev<T>(t);
    Unroll<0, Q>::run([&](auto q) {
        constexpr int j = decltype(q)::value;
        const int w = bitrev<Q>(j) * T + brt;      // frequency of position t Q + j
        const bool cj = w > S;
        const int ws = cj ? P - w : w;
        C h0 = sm.H[ws][i0][line], h1 = sm.H[ws][i1][line], h2 = sm.H[ws][i2][line];
        if (cj) { h0.y = -h0.y; h1.y = -h1.y; h2.y = -h2.y; }
        const int pos = t * Q + j;
        x[j] = cadd(cadd(cmul(h0, sm.X[pos][0][line]), cmul(h1, sm.X[pos][1][line])),
                    cmul(h2, sm.X[pos][2][line]));
    });
    fft_dit_reg<C, Q, T, +1>(x, sm.tw, t);
    if (!live) return;
    const R scale = sig / (R)P;
    // outputs are the last S positions: threads t >= T/2 hold them
    if (t * Q + Q <= S) return;
    Unroll<0, Q>::run([&](auto q) {
        constexpr int j = decltype(q)::value;
        const int pos = t * Q + j;
        if (pos < S) return;
        C v = x[j];
        v.x *= scale; v.y *= scale;
        a.acc[((long long)sm.out[pos - S] * 3 + comp) * a.nbins + row] = v;
    });
}

template <typename R, int Q, int T>
void far_launch_reg(mot_ctx* c, FarArgs<R>& a, cudaStream_t s) {
    typedef FarRegSmem<R, Q, T> SM;
    MOT_CUDA_TRY(cudaFuncSetAttribute(k_far_reg<R, Q, T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM)));
    MOT_CUDA_TRY(cudaFuncSetAttribute(k_far_reg<R, Q, T>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    a.ntile = (c->Hu + SM::NB - 1) / SM::NB;
    const long long blocks = (long long)c->Hw * c->Hv * 4 * a.ntile;
    k_far_reg<R, Q, T><<<(int)blocks, 96, sizeof(SM), s>>>(a);
    MOT_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- four-step variant
// Levels with 2S = P > 32 (FP32) / 16 (FP64): the temporal transform of length
// P = T Q1 is split as n = t + T n2, k = k2 + Q1 k1 (Bailey's four-step form):
//   X[k2 + Q1 k1] = sum_t W_T^{t k1} W_P^{t k2} sum_{n2} x[t + T n2] W_Q1^{n2 k2}.
// Phase A: a thread per (component, bin, t) loads its time-strided subsequence and
//   runs the Q1-point transform in registers (literal twiddles); the results go to
//   shared memory, XOR-swizzled by lane so that the warp's 32 rows hit 32 banks.
// Phase B: an item per (bin, k2) gathers the three components over t, applies
//   W_P^{t k2} (powers of one table root), the T-point transforms, the 3x3 product
//   with the level spectra, the inverse T-point transforms and the conjugate
//   twiddles, and writes back in place.
// Phase C: the thread of phase A runs the inverse Q1-point transform and stores its
//   outputs in the second half of the window (times n0 .. n0 + S - 1).
// A block is 256 threads: phases A and C use 3 NB T = 192 of them, phase B all.
template <typename R, int P> struct Far4 {
    typedef typename CT<R>::c C;
    static constexpr int Q1 = sizeof(R) == 4 ? 32 : 16;
    static constexpr int T = P / Q1;
    static constexpr int NB = (sizeof(R) == 4 ? 2048 : 1024) / P;
    static constexpr int S = P / 2;
    static constexpr int NA = 3 * NB * T;
    static constexpr int NI = NB * Q1;
    static constexpr int NTB = 256;
    static_assert(NA == 192 && T >= 2 && Q1 * T == P, "four-step shape");
    struct Smem {
        C Y[3 * NB * T][Q1];      // row (c NB + bin) T + t, column k2 ^ key(row)
        C H[S + 1][7 * NB];       // level spectra [w][c NB + bin], rows padded by NB
        C tw[Q1];                 // W_P^{k2}
        int in[P];                // ring slot of every window time (-1: none)
        int out[S];               // accumulator slot of every output time
    };
    // phase-A thread of (component, t, bin); its lane (index mod 32) keys the swizzle
    __device__ static int athread(int c, int t, int bin) { return (c * T + t) * NB + bin; }
    __device__ static int row(int c, int t, int bin) { return (c * NB + bin) * T + t; }
    __device__ static int col(int k2, int a) { return k2 ^ (a & (Q1 - 1)); }
};

template <typename R, int P>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k_far_4s(FarArgs<R> a) {
    static_assert(std::is_same<R, double>::value, "FP32 far levels run k_far_fs");
    typedef Far4<R, P> F;
    typedef typename F::C C;
    constexpr int Q1 = F::Q1, T = F::T, NB = F::NB, S = F::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename F::Smem& sm = *reinterpret_cast<typename F::Smem*>(smem_raw);
    const int tid = threadIdx.x;
    const int ut = blockIdx.x % a.ntile;
    const int rest = blockIdx.x / a.ntile;
    const int mirror = rest & 3;
    const int orow = rest >> 2;
    const int kv_o = orow % a.Hv, kw_o = orow / a.Hv;
    const bool fv = (mirror & 1) != 0, fw = (mirror & 2) != 0;
    const bool mv = kv_o > 0 && 2 * kv_o < a.Pv;
    const bool mw = kw_o > 0 && 2 * kw_o < a.Pw;
    if ((fv && !mv) || (fw && !mw)) return;
    const int kv = fv ? a.Pv - kv_o : kv_o;
    const int kw = fw ? a.Pw - kw_o : kw_o;
    const int ku0 = ut * NB;
    const int nlive = min(NB, a.Hu - ku0);
    const long long row0 = ((long long)kw * a.Pv + kv) * a.Hu + ku0;
    const long long obase = ((long long)kw_o * a.Hv + kv_o) * a.Hu + ku0;
    for (int i = tid; i < (S + 1) * 6 * NB; i += F::NTB) {
        const int l = i % NB, wc = i / NB;      // wc = w * 6 + c
        if (l < nlive)
            cp_async_c(&sm.H[wc / 6][(wc % 6) * NB + l], a.H + (long long)wc * a.noct + obase + l);
    }
    const int tfirst = max(1, a.n0 - a.lmax);
    for (int i = tid; i < P; i += F::NTB) {
        const int time = a.w0 + i;
        sm.in[i] = time >= tfirst ? time % a.hring : -1;
        if (i < S) sm.out[i] = (a.n0 + i) % a.smax;
        if (i < Q1) sm.tw[i] = a.tw[i];     // W_P^i
    }
    __syncthreads();
    // ---- phase A
    const int bin = tid % NB, ct = tid / NB;
    const int t = ct % T, comp = ct / T;
    const bool athr = tid < F::NA;
    const bool live = athr && bin < nlive;
    const R sig = comp == 0 ? (R)1 : (comp == 1 ? (fv ? (R)-1 : (R)1) : (fw ? (R)-1 : (R)1));
    C x[Q1];
    if (athr) {
        Unroll<0, Q1>::run([&](auto q) {
            constexpr int n2 = decltype(q)::value;
            const int slot = sm.in[t + T * n2];
            C v;
            v.x = 0; v.y = 0;
            if (slot >= 0 && live) v = a.ring[((long long)slot * 3 + comp) * a.nbins + row0 + bin];
            v.x *= sig; v.y *= sig;
            x[n2] = v;
        });
        fft_dif_reg<C, Q1, 1, -1>(x, sm.tw, 0);      // register j holds k2 = bitrev(j)
        C* yr = sm.Y[F::row(comp, t, bin)];
        Unroll<0, Q1>::run([&](auto q) {
            constexpr int j = decltype(q)::value;
            yr[F::col(bitrev<Q1>(j), tid)] = x[j];
        });
    }
    cp_async_commit_wait();
    __syncthreads();
    // ---- phase B
    for (int it = tid; it < F::NI; it += F::NTB) {
        const int b = it % NB, k2 = it / NB;
        C wt[T];                                 // W_P^{t k2}
        wt[0].x = 1; wt[0].y = 0;
        wt[1] = sm.tw[k2];
        Unroll<2, T>::run([&](auto q) {
            constexpr int tt = decltype(q)::value;
            wt[tt] = cmul(wt[tt - 1], wt[1]);
        });
        C v[3][T];
        Unroll<0, 3>::run([&](auto cq) {
            constexpr int c = decltype(cq)::value;
            Unroll<0, T>::run([&](auto q) {
                constexpr int tt = decltype(q)::value;
                v[c][tt] = cmul(sm.Y[F::row(c, tt, b)][F::col(k2, F::athread(c, tt, b))], wt[tt]);
            });
            fft_dif_reg<C, T, 1, -1>(v[c], sm.tw, 0);   // register j holds k1 = bitrev(j)
        });
        Unroll<0, T>::run([&](auto q) {
            constexpr int j = decltype(q)::value;
            const int w = k2 + Q1 * bitrev<T>(j);
            const bool cj = w > S;
            const int ws = cj ? P - w : w;
            const C* hp = &sm.H[ws][b];
            C h[6];
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) {
                h[cc] = hp[cc * NB];
                if (cj) h[cc].y = -h[cc].y;
            }
            const C x0 = v[0][j], x1 = v[1][j], x2 = v[2][j];
            v[0][j] = cadd(cadd(cmul(h[0], x0), cmul(h[3], x1)), cmul(h[4], x2));
            v[1][j] = cadd(cadd(cmul(h[3], x0), cmul(h[1], x1)), cmul(h[5], x2));
            v[2][j] = cadd(cadd(cmul(h[4], x0), cmul(h[5], x1)), cmul(h[2], x2));
        });
        Unroll<0, 3>::run([&](auto cq) {
            constexpr int c = decltype(cq)::value;
            fft_dit_reg<C, T, 1, +1>(v[c], sm.tw, 0);   // register t holds C_t
            Unroll<0, T>::run([&](auto q) {
                constexpr int tt = decltype(q)::value;
                C w = wt[tt];
                w.y = -w.y;
                sm.Y[F::row(c, tt, b)][F::col(k2, F::athread(c, tt, b))] = cmul(v[c][tt], w);
            });
        });
    }
    __syncthreads();
    // ---- phase C
    if (!live) return;
    const C* yr = sm.Y[F::row(comp, t, bin)];
    Unroll<0, Q1>::run([&](auto q) {
        constexpr int j = decltype(q)::value;
        x[j] = yr[F::col(bitrev<Q1>(j), tid)];
    });
    fft_dit_reg<C, Q1, 1, +1>(x, sm.tw, 0);          // register n2 holds y[t + T n2]
    const R scale = sig / (R)P;
    Unroll<Q1 / 2, Q1>::run([&](auto q) {
        constexpr int n2 = decltype(q)::value;
        const int pos = t + T * n2;                  // >= S
        C v = x[n2];
        v.x *= scale; v.y *= scale;
        a.acc[((long long)sm.out[pos - S] * 3 + comp) * a.nbins + row0 + bin] = v;
    });
}

template <typename R, int P>
void far_launch_4s(mot_ctx* c, FarArgs<R>& a, cudaStream_t s) {
    typedef Far4<R, P> F;
    const int sm_bytes = (int)sizeof(typename F::Smem);
    MOT_CUDA_TRY(cudaFuncSetAttribute(k_far_4s<R, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      sm_bytes));
    MOT_CUDA_TRY(cudaFuncSetAttribute(k_far_4s<R, P>,
                                      cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    a.ntile = (c->Hu + F::NB - 1) / F::NB;
    const long long blocks = (long long)c->Hw * c->Hv * 4 * a.ntile;
    k_far_4s<R, P><<<(int)blocks, F::NTB, sm_bytes, s>>>(a);
    MOT_LAUNCH_CHECK();
}

template <typename R, int TB>
void far_launch(mot_ctx* c, FarArgs<R>& a, cudaStream_t s) {
    typedef typename CT<R>::c C;
    a.ntile = (c->Hu + TB - 1) / TB;
    const int P = 2 * a.S;
    const size_t sm = sizeof(C) * ((size_t)tw_entries<C>(P) + 2 * (size_t)P * (3 * TB + 1));
    if (sm > 220 * 1024 || a.S > kMaxLevel)
        throw MotError{MOT_ERR_ARG, "blocked scheme: level too long for shared memory"};
    // the limit is process-wide and P varies by level and context: set the device's
    // opt-in maximum (never lowered by another launch), the need is checked above
    int dev = 0, optin = 0;
    MOT_CUDA_TRY(cudaGetDevice(&dev));
    MOT_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (sm > (size_t)optin)
        throw MotError{MOT_ERR_ARG, "blocked scheme: level too long for shared memory"};
    MOT_CUDA_TRY(cudaFuncSetAttribute(k_far<R, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MOT_CUDA_TRY(cudaFuncSetAttribute(k_far<R, TB>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    const long long blocks = (long long)c->Hw * c->Hv * 4 * a.ntile;
    k_far<R, TB><<<(int)blocks, NT, sm, s>>>(a);
    MOT_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- FP32 far levels
// The block product of one level firing with the four-step transform of length
// P = Q1 T (Q1 = 16, T = P / 16 = 1 .. 16) in which every thread holds all three
// components of its share of a temporal line: the 3x3 product then needs no exchange
// between components, and every thread works in every phase.
//   phase A: thread (t, bin) loads x[t + T n2], n2 < 16, of the three components (the
//            window times w0 + t + T n2; zero before tfirst), runs the 16-point
//            DFTs in registers (compile-time twiddles), multiplies by W_P^{t k2} and
//            stores to shared memory;
//   phase B: thread (tt, bin) takes k2 = tt, tt + T, ...: the T values of each
//            component, T-point DFTs (frequency w = k2 + 16 k1), the 3x3 product with
//            the level spectrum H(w) ([w][6][octant bin] in global memory, coalesced
//            over consecutive bins; conj H(P - w) above S), inverse T-point DFTs and
//            W_P^{-t k2}, back to shared memory;
//   phase C: thread (t, bin) runs the inverse 16-point DFTs over k2 and stores
//            y[t + T n2] for n2 >= 8, the last S = 8 T positions of the window.
// With T = 1 (P = 16) one thread per bin does all of it in registers.  A CTA takes
// NB = 128 / T consecutive octant bins (across rfft rows) and walks the four mirror
// rows (ku, +-kv, +-kw) of each; a mirror that does not exist for a bin's row
// (kv = 0 or Pv / 2, likewise kw) only skips that bin's loads and stores.  The level
// spectra of the CTA's bins are staged in shared memory once for the four mirrors
// (they were the loads the product waited on), and for T > 1 the next mirror's window
// is loaded into the phase-A registers while phases B and C of the current one run.  Mirror
// signs: inputs and outputs of component b are scaled by sigma_b (sigma_x = 1,
// sigma_y = -1 on a mirrored v, sigma_z = -1 on a mirrored w), so the octant spectra
// serve every mirror.  Shared memory element (c, k2, t, bin) sits at
// c CS + k2 KS + t NB + bin, KS padded for NB = 8 so that no phase has bank conflicts.
template <int P> struct FarFS {
    static constexpr int Q1 = 16, T = P / Q1, S = P / 2, NTH = 128, NB = NTH / T;
    static constexpr int KS = T * NB + (NB < 16 ? 8 : 0);
    static constexpr int CS = Q1 * KS;
    static_assert(T >= 1 && T * Q1 == P && T <= 16, "far four-step shape");
    // the level spectra of the CTA's bins, [w][c][bin], staged once for the four
    // mirrors (copied asynchronously while the first window loads); rows of one
    // frequency padded when NB = 8, where the lanes of a half-warp read two frequencies
    static constexpr int HW = 6 * NB + (NB < 16 ? 8 : 0);
    static constexpr int HS = (S + 1) * HW;
    struct Smem {
        float2 V[T > 1 ? 3 * CS : 2];
        float2 H[HS];
        float2 tw[P];          // W_P^m, m < P (the FP32 table's hi parts)
        int in[P];             // ring slot of every window time (-1: none)
        int out[S];            // accumulator slot of every output time
    };
};

template <int P>
__global__ void __launch_bounds__(128, P <= 16 ? 4 : 2) k_far_fs(FarArgs<float> a) {
    typedef FarFS<P> F;
    constexpr int Q1 = F::Q1, T = F::T, S = F::S, NB = F::NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename F::Smem& sm = *reinterpret_cast<typename F::Smem*>(smem_raw);
    const int tid = threadIdx.x;
    const int bin = tid % NB, t = tid / NB;
    const long long o = (long long)blockIdx.x * NB + bin;       // octant bin
    const bool obin = o < a.noct;
    const int ku = obin ? (int)(o % a.Hu) : 0;
    const int kv_o = obin ? (int)((o / a.Hu) % a.Hv) : 0;
    const int kw_o = obin ? (int)(o / ((long long)a.Hu * a.Hv)) : 0;
    const bool mv = kv_o > 0 && 2 * kv_o < a.Pv;
    const bool mw = kw_o > 0 && 2 * kw_o < a.Pw;
    const int tfirst = max(1, a.n0 - a.lmax);
    {   // H[w][c][bin] <- a.H[(w * 6 + c) * noct + o0 + bin], o0 the CTA's first bin
        const long long o0 = (long long)blockIdx.x * NB;
        for (int i = tid; i < (S + 1) * 6 * NB; i += F::NTH) {
            const int b = i % NB, wc = i / NB;                 // wc = w * 6 + c
            const bool ok = o0 + b < a.noct;
            cp_async_c(&sm.H[(wc / 6) * F::HW + (wc % 6) * NB + b],
                       ok ? a.H + (long long)wc * a.noct + o0 + b : a.H, ok);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (int i = tid; i < P; i += F::NTH) {
        const int time = a.w0 + i;
        sm.in[i] = time >= tfirst ? time % a.hring : -1;
        sm.tw[i] = a.tw[i];
        if (i < S) sm.out[i] = (a.n0 + i) % a.smax;
    }
    __syncthreads();
    // mirror m of the bin: whether it exists, its rfft bin, the signs sigma_y, sigma_z
    auto mirror_of = [&](int m, bool& live, long long& bidx, float& sy, float& sz) {
        const bool fv = (m & 1) != 0, fw = (m & 2) != 0;
        live = obin && (!fv || mv) && (!fw || mw);
        const int kv = fv ? a.Pv - kv_o : kv_o;
        const int kw = fw ? a.Pw - kw_o : kw_o;
        bidx = ((long long)kw * a.Pv + kv) * a.Hu + ku;
        sy = fv ? -1.f : 1.f;
        sz = fw ? -1.f : 1.f;
    };
    // window samples x[t + T n2], n2 < Q1, of the three components (sigma-scaled)
    auto load_window = [&](int m, float2 (&x)[3][Q1]) {
        bool live;
        long long bidx;
        float sy, sz;
        mirror_of(m, live, bidx, sy, sz);
        Unroll<0, Q1>::run([&](auto q) {
            constexpr int n2 = decltype(q)::value;
            const int slot = sm.in[t + T * n2];
            float2 v0 = make_float2(0.f, 0.f), v1 = v0, v2 = v0;
            if (live && slot >= 0) {
                const float2* src = a.ring + (long long)slot * 3 * a.nbins + bidx;
                v0 = src[0];
                v1 = src[a.nbins];
                v2 = src[2 * a.nbins];
            }
            x[0][n2] = v0;
            x[1][n2] = make_float2(sy * v1.x, sy * v1.y);
            x[2][n2] = make_float2(sz * v2.x, sz * v2.y);
        });
    };
    // outputs y[t + T n2], n2 >= Q1 / 2, i.e. window positions S .. P - 1
    auto store_outputs = [&](int m, float2 (&y)[3][Q1]) {
        bool live;
        long long bidx;
        float sy, sz;
        mirror_of(m, live, bidx, sy, sz);
        if (!live) return;
        const float sc = 1.f / (float)P;
        Unroll<Q1 / 2, Q1>::run([&](auto q) {
            constexpr int n2 = decltype(q)::value;
            const int pos = t + T * n2;                      // >= S
            float2* dst = a.acc + (long long)sm.out[pos - S] * 3 * a.nbins + bidx;
            dst[0] = make_float2(sc * y[0][n2].x, sc * y[0][n2].y);
            dst[a.nbins] = make_float2(sy * sc * y[1][n2].x, sy * sc * y[1][n2].y);
            dst[2 * a.nbins] = make_float2(sz * sc * y[2][n2].x, sz * sc * y[2][n2].y);
        });
    };
    float2 x[3][Q1];
    if constexpr (T > 1) load_window(0, x);
    for (int mirror = 0; mirror < 4; ++mirror) {
        if constexpr (T == 1) load_window(mirror, x);
        Unroll<0, 3>::run([&](auto cq) { dft_ct<Q1, -1>(x[decltype(cq)::value]); });
        if constexpr (T == 1) {
            // ---- the whole product in registers: frequency w = k2
            if (mirror == 0) {
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                __syncthreads();
            }
            Unroll<0, Q1>::run([&](auto q) {
                constexpr int w = decltype(q)::value;
                constexpr bool cj = w > S;
                constexpr int ws = cj ? P - w : w;
                float2 h[6];
#pragma unroll
                for (int cc = 0; cc < 6; ++cc) {
                    h[cc] = sm.H[ws * F::HW + cc * NB + bin];
                    if (cj) h[cc].y = -h[cc].y;
                }
                const float2 x0 = x[0][w], x1 = x[1][w], x2 = x[2][w];
                x[0][w] = cadd(cadd(cmul(h[0], x0), cmul(h[3], x1)), cmul(h[4], x2));
                x[1][w] = cadd(cadd(cmul(h[3], x0), cmul(h[1], x1)), cmul(h[5], x2));
                x[2][w] = cadd(cadd(cmul(h[4], x0), cmul(h[5], x1)), cmul(h[2], x2));
            });
            Unroll<0, 3>::run([&](auto cq) { dft_ct<Q1, +1>(x[decltype(cq)::value]); });
            store_outputs(mirror, x);
        } else {
            // ---- phase A (the DFTs over n2 above), twiddles W_P^{t k2}, exchange
            Unroll<0, Q1>::run([&](auto q) {
                constexpr int k2 = decltype(q)::value;
                // the four-step twiddles as plain FP32 values: unlike the DFT
                // constants they hardly change the march (6.3e-6 against 5.8e-6 with
                // float pairs, 32^3 sphere), at 2 % of the step time
                const float2 w = sm.tw[t * k2];
                float2* dst = &sm.V[k2 * F::KS + t * NB + bin];
                dst[0] = cmul(x[0][k2], w);
                dst[F::CS] = cmul(x[1][k2], w);
                dst[2 * F::CS] = cmul(x[2][k2], w);
            });
            if (mirror == 0) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            __syncthreads();
            // the next mirror's window streams in while phases B and C of this one run
            if (mirror < 3) load_window(mirror + 1, x);
            // ---- phase B: T-point DFTs over t, product, inverse, conjugate twiddles
            for (int j = 0; j < Q1 / T; ++j) {
                const int k2 = t + T * j;
                float2 v[3][T];
                Unroll<0, T>::run([&](auto q) {
                    constexpr int tt = decltype(q)::value;
                    const float2* src = &sm.V[k2 * F::KS + tt * NB + bin];
                    v[0][tt] = src[0];
                    v[1][tt] = src[F::CS];
                    v[2][tt] = src[2 * F::CS];
                });
                Unroll<0, 3>::run([&](auto cq) { dft_ct<T, -1>(v[decltype(cq)::value]); });
                Unroll<0, T>::run([&](auto q) {
                    constexpr int k1 = decltype(q)::value;
                    const int w = k2 + Q1 * k1;
                    const bool cj = w > S;
                    const int ws = cj ? P - w : w;
                    float2 h[6];
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) {
                        h[cc] = sm.H[ws * F::HW + cc * NB + bin];
                        if (cj) h[cc].y = -h[cc].y;
                    }
                    const float2 x0 = v[0][k1], x1 = v[1][k1], x2 = v[2][k1];
                    v[0][k1] = cadd(cadd(cmul(h[0], x0), cmul(h[3], x1)), cmul(h[4], x2));
                    v[1][k1] = cadd(cadd(cmul(h[3], x0), cmul(h[1], x1)), cmul(h[5], x2));
                    v[2][k1] = cadd(cadd(cmul(h[4], x0), cmul(h[5], x1)), cmul(h[2], x2));
                });
                Unroll<0, 3>::run([&](auto cq) { dft_ct<T, +1>(v[decltype(cq)::value]); });
                Unroll<0, T>::run([&](auto q) {
                    constexpr int tt = decltype(q)::value;
                    const float2 w = cconj(sm.tw[tt * k2]);
                    float2* dst = &sm.V[k2 * F::KS + tt * NB + bin];
                    dst[0] = cmul(v[0][tt], w);
                    dst[F::CS] = cmul(v[1][tt], w);
                    dst[2 * F::CS] = cmul(v[2][tt], w);
                });
            }
            __syncthreads();
            // ---- phase C: gather over k2, inverse DFTs over k2, stores
            float2 y[3][Q1];
            Unroll<0, Q1>::run([&](auto q) {
                constexpr int k2 = decltype(q)::value;
                const float2* src = &sm.V[k2 * F::KS + t * NB + bin];
                y[0][k2] = src[0];
                y[1][k2] = src[F::CS];
                y[2][k2] = src[2 * F::CS];
            });
            __syncthreads();   // the next mirror's phase A overwrites V
            Unroll<0, 3>::run([&](auto cq) { dft_ct<Q1, +1>(y[decltype(cq)::value]); });
            store_outputs(mirror, y);
        }
    }
}

template <int P>
void far_launch_fs(mot_ctx* c, FarArgs<float>& a, cudaStream_t s) {
    typedef FarFS<P> F;
    const int sm_bytes = (int)sizeof(typename F::Smem);
    MOT_CUDA_TRY(cudaFuncSetAttribute(k_far_fs<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      sm_bytes));
    MOT_CUDA_TRY(cudaFuncSetAttribute(k_far_fs<P>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      100));
    const long long blocks = (c->noct + F::NB - 1) / F::NB;
    k_far_fs<P><<<(int)blocks, F::NTH, sm_bytes, s>>>(a);
    MOT_LAUNCH_CHECK();
}

template <typename R>
void far_level(mot_ctx* c, int k, int n0, cudaStream_t s) {
    HistoryBuffers<R>& hb = hbuf<R>(c);
    FarArgs<R> a;
    a.ring = hb.jhat_ring;
    a.hring = c->hring;
    a.nbins = c->nbins;
    a.noct = c->noct;
    a.H = hb.level_spec + c->lev_off[k];
    a.acc = hb.acc_ring + c->lev_acc[k] * 3 * c->nbins;
    a.smax = c->lev_S[k];
    a.n0 = n0;
    a.S = c->lev_S[k];
    a.lmax = std::min(c->lev_a[k] + a.S - 1, c->ell);
    a.w0 = n0 - c->lev_a[k] - a.S;
    a.Hu = c->Hu; a.Hv = c->Hv; a.Hw = c->Hw;
    a.Pv = c->ax[1].P; a.Pw = c->ax[2].P;
    const AxisFFT& f = c->lev_fft[k];
    a.rl.P = f.P;
    a.rl.n = f.nrad;
    for (int i = 0; i < 16; ++i) a.rl.r[i] = f.rad[i];
    a.tw = twtab<R>(f);
    // lines per CTA: 3 components x TB bins; fewer bins for long levels keeps several
    // CTAs resident per SM
    // lines of up to 32 (FP32) / 16 (FP64) points: one thread per line, in registers;
    // longer lines: the four-step kernel (FP64 S = 128: lines split over 8 lanes with
    // shuffle stages); beyond S = 128 the shared-memory Stockham kernel
    if constexpr (std::is_same<R, float>::value) {
        switch (a.S) {
            case 2: far_launch_reg<R, 4, 1>(c, a, s); break;
            case 4: far_launch_reg<R, 8, 1>(c, a, s); break;
            case 8: far_launch_fs<16>(c, a, s); break;
            case 16: far_launch_fs<32>(c, a, s); break;
            case 32: far_launch_fs<64>(c, a, s); break;
            case 64: far_launch_fs<128>(c, a, s); break;
            case 128: far_launch_fs<256>(c, a, s); break;
            default: far_launch<R, 4>(c, a, s);
        }
    } else {
        switch (a.S) {
            case 2: far_launch_reg<R, 4, 1>(c, a, s); break;
            case 4: far_launch_reg<R, 8, 1>(c, a, s); break;
            case 8: far_launch_reg<R, 16, 1>(c, a, s); break;
            case 16: far_launch_4s<R, 32>(c, a, s); break;
            case 32: far_launch_4s<R, 64>(c, a, s); break;
            case 64: far_launch_4s<R, 128>(c, a, s); break;
            case 128: far_launch_reg<R, 32, 8>(c, a, s); break;
            default: far_launch<R, 2>(c, a, s);
        }
    }
    c->stats.launches += 1;
    c->stats.far_launches += 1;
}

// hist_spatial <- sum_{l=1}^{ell} G_l * J_{n-l}; J_{n-1} is read from the spatial ring
template <typename R>
void history_step(mot_ctx* c, int n, cudaStream_t s, cudaEvent_t* ev) {
    typedef typename CT<R>::c C;
    HistoryBuffers<R>& hb = hbuf<R>(c);
    const long long slot = 3 * c->nbins;
    if (n >= 2) {
        const double* Jprev = c->J + slot_index(n - 1, c->jring) * 3 * c->M;
        fft_forward<R>(c, Jprev, hb.jhat_ring + slot_index(n - 1, c->hring) * slot, s,
                       c->adjoint ? c->chi : nullptr);
        c->stats.launches += 3;
    }
    if (ev) MOT_CUDA_TRY(cudaEventRecord(ev[0], s));
    const bool blocked = c->scheme == MOT_HISTORY_BLOCKED;
    if (blocked)   // each firing level writes its own accumulator ring
        for (int k = c->nlev - 1; k >= 0; --k)
            if ((n - 1) % c->lev_S[k] == 0) far_level<R>(c, k, n, s);
    if (ev) MOT_CUDA_TRY(cudaEventRecord(ev[1], s));
    const R scale = (R)(1.0 / ((double)c->ax[0].P * c->ax[1].P * c->ax[2].P));
    const long long nblk = (c->noct + 8 * (NT / 32) - 1) / (8 * (NT / 32));
    const int L = blocked ? std::min(c->block - 1, c->ell) : c->ell;
    FarSums<C> far;
    far.n = blocked ? c->nlev : 0;
    for (int k = 0; k < far.n; ++k)
        far.p[k] = hb.acc_ring + (c->lev_acc[k] + slot_index(n, c->lev_S[k])) * slot;
    k_mac<R><<<(int)nblk, NT, 0, s>>>(hb.ghat, hb.jhat_ring, c->hring,
                                      (int)slot_index(n - 1, c->hring), L, geom(c), scale,
                                      hb.phat, far);
    MOT_LAUNCH_CHECK();
    c->stats.launches += 1;
    c->stats.mac_launches += 1;
    if (ev) MOT_CUDA_TRY(cudaEventRecord(ev[2], s));
    fft_inverse<R>(c, hb.phat, hb.hist_spatial, s);
    c->stats.launches += 3;
}

template void history_alloc<double>(mot_ctx*);
template void history_alloc<float>(mot_ctx*);
template void history_alloc_shared<double>(mot_ctx*, mot_ctx*);
template void history_alloc_shared<float>(mot_ctx*, mot_ctx*);
template void history_free<double>(mot_ctx*);
template void history_free<float>(mot_ctx*);
template void history_reset<double>(mot_ctx*, cudaStream_t);
template void history_reset<float>(mot_ctx*, cudaStream_t);
template void level_spectra<double>(mot_ctx*);
template void level_spectra<float>(mot_ctx*);
template void history_step<double>(mot_ctx*, int, cudaStream_t, cudaEvent_t*);
template void history_step<float>(mot_ctx*, int, cudaStream_t, cudaEvent_t*);

}  // namespace mot

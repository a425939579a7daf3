// Spatial spectra of the interaction elements (App. A, Sec. 3).
//
// The product G_l * J over the N-voxel grid is a 3-level block-Toeplitz product.
// Embedded in a circulant of size P >= 2N - 1 per axis (App. A), it becomes a
// pointwise product of DFTs, with the kernel's DFT
//     Ghat_l(k) = sum_{d = -(N-1)}^{N-1} G_l(d) exp(-2 pi i k . d / P).
// G is even in every d_i for the diagonal components and odd in d_a, d_b (even in the
// third) for the (a, b) component, so Ghat is real, has the same parity in k, and is
// a product of one-sided cosine / sine sums along each axis:
//     even axis: sum_{d>=0} c_d G(d) cos(2 pi k d / P),  c_0 = 1, c_{d>0} = 2
//     odd axis:  sum_{d>0} 2 G(d) sin(2 pi k d / P) times -i; two odd axes give -1.
// Only the octant k_i in [0, P_i/2] is stored; the other bins follow by parity.
#include "mot_internal.cuh"

#include <algorithm>

namespace {

// trig tables laid out [d][k] (k fastest), k < H = P/2 + 1, d < N
__global__ void trig_table_kernel(int P, int N, int H, double* cosw, double* sinw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * H) return;
    const int d = i / H, k = i % H;
    const long long kd = ((long long)k * d) % P;
    double s, c;
    sincospi(2.0 * (double)kd / (double)P, &s, &c);
    cosw[i] = (d == 0 ? 1.0 : 2.0) * c;
    sinw[i] = (d == 0 ? 0.0 : 2.0) * s;
}

__global__ void extract_lag_kernel(const int* __restrict__ tab_l0, const double* __restrict__ tab,
                                   long long noff, int l, int cc, double* __restrict__ g) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= noff) return;
    const int idx = l - tab_l0[i];
    g[i] = (idx >= 0 && idx < mot::WIN) ? tab[(i * 6 + cc) * mot::WIN + idx] : 0.0;
}

// g[d] = sum_{l <= n} w[l] G_l(d) for component cc (the lags of the window at d)
__global__ void extract_weighted_kernel(const int* __restrict__ tab_l0,
                                        const double* __restrict__ tab, long long noff,
                                        const double* __restrict__ w, int n, int cc,
                                        double* __restrict__ g) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= noff) return;
    const int l0 = tab_l0[i];
    double acc = 0.0;
    for (int k = 0; k < mot::WIN && l0 + k <= n; ++k)
        if (l0 + k >= 0) acc = fma(w[l0 + k], tab[(i * 6 + cc) * mot::WIN + k], acc);
    g[i] = acc;
}

// dst[o][cc] += w * src[cc][o], src optionally rounded to FP32 first
__global__ void accum_kernel(const double* __restrict__ src, long long noct, double w,
                             int round32, double* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * noct) return;
    const long long o = i / 6;
    const int cc = (int)(i % 6);
    double v = src[cc * noct + o];
    if (round32) v = (double)(float)v;
    dst[i] = fma(w, v, dst[i]);
}

// out[o2][o1][k] = sum_{d < n} in[o2][o1][d] * w[d][k]         (transform along the fastest axis)
__global__ void pass_fast(const double* __restrict__ in, int n, long long nrows,
                          const double* __restrict__ w, int K, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows * K) return;
    const long long row = i / K;
    const int k = (int)(i % K);
    const double* src = in + row * n;
    double acc = 0.0;
    for (int d = 0; d < n; ++d) acc = fma(src[d], w[(long long)d * K + k], acc);
    out[i] = acc;
}

// out[o][k][f] = sum_{d < n} in[o][d][f] * w[d][k]           (transform along a middle axis)
__global__ void pass_mid(const double* __restrict__ in, int n, int F, long long nouter,
                         const double* __restrict__ w, int K, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nouter * K * F) return;
    const int f = (int)(i % F);
    const int k = (int)((i / F) % K);
    const long long o = i / ((long long)F * K);
    const double* src = in + o * (long long)n * F + f;
    double acc = 0.0;
    for (int d = 0; d < n; ++d) acc = fma(src[(long long)d * F], w[(long long)d * K + k], acc);
    out[i] = acc;
}

// [6][noct] (component-major) -> [noct][6] in the history precision
template <typename R>
__global__ void interleave_kernel(const double* __restrict__ src, long long noct,
                                  R* __restrict__ dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * noct) return;
    const long long o = i / 6;
    const int cc = (int)(i % 6);
    dst[i] = (R)src[cc * noct + o];
}

// x[i] *= s (in place)
__global__ void scale_inplace_kernel(double* x, long long n, double s) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] *= s;
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

struct TrigTables {
    double* cosw[3] = {nullptr, nullptr, nullptr};
    double* sinw[3] = {nullptr, nullptr, nullptr};
    ~TrigTables() {
        for (int a = 0; a < 3; ++a) { cudaFree(cosw[a]); cudaFree(sinw[a]); }
    }
};

struct Scratch {
    double* g = nullptr;
    double* t1 = nullptr;
    double* t2 = nullptr;
    ~Scratch() { cudaFree(g); cudaFree(t1); cudaFree(t2); }
};

// odd axes of component cc (order xx, yy, zz, xy, xz, yz): bit a set if odd along a
const int kOddMask[6] = {0, 0, 0, 3, 5, 6};

// spectrum of the octant kernel sc.g (component cc) into dst [noct]
void transform_one(mot_ctx* c, const TrigTables& tt, Scratch& sc, int cc, double* dst) {
    const int U = c->U, V = c->V, W = c->W;
    const int Hu = c->Hu, Hv = c->Hv, Hw = c->Hw;
    cudaStream_t s = c->stream;
    const int odd = kOddMask[cc];
    const double* wx = (odd & 1) ? tt.sinw[0] : tt.cosw[0];
    const double* wy = (odd & 2) ? tt.sinw[1] : tt.cosw[1];
    const double* wz = (odd & 4) ? tt.sinw[2] : tt.cosw[2];
    // x: [W][V][U] -> [W][V][Hu]
    pass_fast<<<nblk((long long)W * V * Hu, 256), 256, 0, s>>>(sc.g, U, (long long)W * V, wx, Hu, sc.t1);
    MOT_LAUNCH_CHECK();
    // y: [W][V][Hu] -> [W][Hv][Hu]
    pass_mid<<<nblk((long long)W * Hv * Hu, 256), 256, 0, s>>>(sc.t1, V, Hu, W, wy, Hv, sc.t2);
    MOT_LAUNCH_CHECK();
    // z: [W][Hv*Hu] -> [Hw][Hv*Hu]
    pass_mid<<<nblk((long long)Hw * Hv * Hu, 256), 256, 0, s>>>(sc.t2, W, Hv * Hu, 1, wz, Hw, dst);
    MOT_LAUNCH_CHECK();
    if (odd) {   // two odd axes: (-i)(-i) = -1
        scale_inplace_kernel<<<nblk(c->noct, 256), 256, 0, s>>>(dst, c->noct, -1.0);
        MOT_LAUNCH_CHECK();
    }
}

void spectrum_one(mot_ctx* c, const TrigTables& tt, Scratch& sc, int l, int cc, double* dst) {
    const long long noff = (long long)c->U * c->V * c->W;
    extract_lag_kernel<<<nblk(noff, 256), 256, 0, c->stream>>>(c->tab_l0, c->tab, noff, l, cc,
                                                              sc.g);
    MOT_LAUNCH_CHECK();
    transform_one(c, tt, sc, cc, dst);
}

void make_tables(mot_ctx* c, TrigTables& tt) {
    const int N[3] = {c->U, c->V, c->W};
    const int H[3] = {c->Hu, c->Hv, c->Hw};
    for (int a = 0; a < 3; ++a) {
        MOT_CUDA_TRY(cudaMalloc(&tt.cosw[a], sizeof(double) * N[a] * H[a]));
        MOT_CUDA_TRY(cudaMalloc(&tt.sinw[a], sizeof(double) * N[a] * H[a]));
        trig_table_kernel<<<nblk((long long)N[a] * H[a], 256), 256, 0, c->stream>>>(
            c->ax[a].P, N[a], H[a], tt.cosw[a], tt.sinw[a]);
        MOT_LAUNCH_CHECK();
    }
}

void make_scratch(mot_ctx* c, Scratch& sc) {
    const long long noff = (long long)c->U * c->V * c->W;
    MOT_CUDA_TRY(cudaMalloc(&sc.g, sizeof(double) * noff));
    MOT_CUDA_TRY(cudaMalloc(&sc.t1, sizeof(double) * (long long)c->W * c->V * c->Hu));
    MOT_CUDA_TRY(cudaMalloc(&sc.t2, sizeof(double) * (long long)c->W * c->Hv * c->Hu));
}

}  // namespace

namespace mot {

// ghat[lag-1][octant bin][6] for lags 1..ell, in the history precision, unnormalised
void compute_spectra(mot_ctx* c) {
    TrigTables tt;
    Scratch sc;
    make_tables(c, tt);
    make_scratch(c, sc);
    double* tmp = nullptr;
    MOT_CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * c->noct * 6));
    try {
        for (int l = 1; l <= c->ell; ++l) {
            for (int cc = 0; cc < 6; ++cc) spectrum_one(c, tt, sc, l, cc, tmp + cc * c->noct);
            const long long off = (long long)(l - 1) * 6 * c->noct;
            if (c->precision == MOT_FP64)
                interleave_kernel<double><<<nblk(6 * c->noct, 256), 256, 0, c->stream>>>(
                    tmp, c->noct, c->h64.ghat + off);
            else
                interleave_kernel<float><<<nblk(6 * c->noct, 256), 256, 0, c->stream>>>(
                    tmp, c->noct, c->h32.ghat + off);
            MOT_LAUNCH_CHECK();
        }
        MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    } catch (...) {
        cudaFree(tmp);
        throw;
    }
    cudaFree(tmp);
}

void spectrum_of_lag(mot_ctx* c, int l, double* host_out) {
    TrigTables tt;
    Scratch sc;
    make_tables(c, tt);
    make_scratch(c, sc);
    double* tmp = nullptr;
    MOT_CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * c->noct * 6));
    try {
        for (int cc = 0; cc < 6; ++cc) spectrum_one(c, tt, sc, l, cc, tmp + cc * c->noct);
        MOT_CUDA_TRY(cudaMemcpyAsync(host_out, tmp, sizeof(double) * c->noct * 6,
                                     cudaMemcpyDeviceToHost, c->stream));
        MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    } catch (...) {
        cudaFree(tmp);
        throw;
    }
    cudaFree(tmp);
}


// dst [noct][6] (FP64, unnormalised) = spectrum of sum_{l=0}^{n} w_l G_l.  Without
// round32 the weighted kernel is combined in space and transformed once; with round32
// every lag l >= 1 is transformed alone and rounded to FP32 before it is weighted (the
// per-lag spectra the FP32-history direct scheme multiplies; lag 0 stays FP64, as in
// the Z_0 solve).
void spectrum_of_combination(mot_ctx* c, const double* w_host, int n, bool round32,
                             double* dst) {
    TrigTables tt;
    Scratch sc;
    make_tables(c, tt);
    make_scratch(c, sc);
    double* tmp = nullptr;
    double* w = nullptr;
    const long long noff = (long long)c->U * c->V * c->W;
    cudaStream_t s = c->stream;
    try {
        MOT_CUDA_TRY(cudaMalloc(&tmp, sizeof(double) * c->noct * 6));
        MOT_CUDA_TRY(cudaMalloc(&w, sizeof(double) * (n + 1)));
        MOT_CUDA_TRY(cudaMemcpyAsync(w, w_host, sizeof(double) * (n + 1),
                                     cudaMemcpyHostToDevice, s));
        if (!round32) {
            for (int cc = 0; cc < 6; ++cc) {
                extract_weighted_kernel<<<nblk(noff, 256), 256, 0, s>>>(c->tab_l0, c->tab, noff,
                                                                       w, n, cc, sc.g);
                MOT_LAUNCH_CHECK();
                transform_one(c, tt, sc, cc, tmp + cc * c->noct);
            }
            interleave_kernel<double><<<nblk(6 * c->noct, 256), 256, 0, s>>>(tmp, c->noct, dst);
            MOT_LAUNCH_CHECK();
        } else {
            MOT_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(double) * 6 * c->noct, s));
            for (int l = 0; l <= n; ++l) {
                if (w_host[l] == 0.0) continue;
                for (int cc = 0; cc < 6; ++cc) spectrum_one(c, tt, sc, l, cc, tmp + cc * c->noct);
                accum_kernel<<<nblk(6 * c->noct, 256), 256, 0, s>>>(tmp, c->noct, w_host[l],
                                                                    l >= 1, dst);
                MOT_LAUNCH_CHECK();
            }
        }
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
    } catch (...) {
        cudaFree(tmp);
        cudaFree(w);
        throw;
    }
    cudaFree(tmp);
    cudaFree(w);
}

}  // namespace mot

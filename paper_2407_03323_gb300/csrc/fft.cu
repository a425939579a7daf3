// Zero-padded 3D FFTs of the current densities and of the history spectrum
// (Sec. 3, Eq. PnFFTMOT; App. A: a Toeplitz product becomes a circulant one after
// zero-padding to P >= n_row + n_col - 1 per axis).
//
// Layouts (per component, 3 components stacked):
//   spatial   [W][V][U]        u fastest (m = u + U (v + V w), Sec. 2.2)
//   after x   [W][V][Hu]       Hu = Pu/2 + 1 (real-to-complex along u)
//   after y   [W][Pv][Hu]
//   spectrum  [Pw][Pv][Hu]
// Forward: three passes x (r2c of paired real rows), y, z; every pass reads only the
// nonzero (unpadded) inputs.  Inverse: z, y, x (c2r), storing only the N outputs the
// grid needs.  Each pass runs batched length-P transforms in shared memory: a CTA
// holds a tile of TB lines as buf[j * (TB+1) + t] and runs mixed-radix Stockham
// stages (radices 2, 3, 4, 5, 7) over it.  Twiddles come from a table of
// exp(-2 pi i k / P) built once per axis with sincospi.  No normalisation is applied.
#include "mot_internal.cuh"

#include <algorithm>

#include "fft_core.cuh"

using namespace mot_fft;

namespace {

constexpr int NT = 256;
constexpr int kLoadBatch = 8;   // global loads a thread keeps in flight while staging a tile

// lines per CTA: 8 (FP64) / 16 (FP32) keeps the shared tile near 60 KB at P = 210,
// so that several CTAs are resident per SM
template <typename R> struct Tile { static constexpr int TB = 8; };
template <> struct Tile<float> { static constexpr int TB = 16; };

// ------------------------------------------------------------------ pass x, forward
// rows (comp, w, v) of a real [3][W][V][U] array, paired (v, v+1) -> [3][W][V][Hu]
template <typename R>
__global__ void __launch_bounds__(NT) k_fwd_x(const double* __restrict__ in, int U, int V, int W,
                                              typename CT<R>::c* __restrict__ out,
                                              const typename CT<R>::c* __restrict__ tw,
                                              RadixList rl, const double* __restrict__ scale) {
    typedef typename CT<R>::c C;
    constexpr int TB = Tile<R>::TB;
    constexpr int ld = TB + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* stw = reinterpret_cast<C*>(smem_raw);
    C* b0 = stw + tw_entries<C>(rl.P);
    C* b1 = b0 + rl.P * ld;
    const int P = rl.P, Hu = P / 2 + 1;
    const int VP = (V + 1) / 2;
    const long long npairs = 3LL * W * VP;
    const long long pair0 = (long long)blockIdx.x * TB;
    load_tw(stw, tw, P);
    // load: z = a + i b, zero-padded; batches of kLoadBatch loads in flight per thread
    for (int it0 = threadIdx.x; it0 < TB * P; it0 += kLoadBatch * blockDim.x) {
        double va[kLoadBatch], vb[kLoadBatch];
#pragma unroll
        for (int q = 0; q < kLoadBatch; ++q) {
            const int it = it0 + q * blockDim.x;
            const int t = it / P, j = it % P;
            const long long pr = pair0 + t;
            va[q] = 0.0;
            vb[q] = 0.0;
            if (it < TB * P && pr < npairs && j < U) {
                const long long cw = pr / VP;
                const int v = (int)(pr % VP) * 2;
                const double* row = in + (cw * V + v) * (long long)U;
                va[q] = row[j];
                if (v + 1 < V) vb[q] = row[U + j];
                if (scale) {   // per-voxel factor (the adjoint transforms chi * lambda)
                    const long long m0 = ((cw % W) * V + v) * (long long)U + j;
                    va[q] *= scale[m0];
                    if (v + 1 < V) vb[q] *= scale[m0 + U];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kLoadBatch; ++q) {
            const int it = it0 + q * blockDim.x;
            if (it >= TB * P) break;
            const int t = it / P, j = it % P;
            C z;
            z.x = (R)va[q];
            z.y = (R)vb[q];
            b0[j * ld + t] = z;
        }
    }
    __syncthreads();
    C* res = fft_tile<C, TB>(b0, b1, P, rl.r, rl.n, ld, stw, -1);
    // split: A = (Z[k] + conj Z[P-k]) / 2, B = -i (Z[k] - conj Z[P-k]) / 2
    for (int it = threadIdx.x; it < TB * Hu; it += blockDim.x) {
        const int t = it / Hu, k = it % Hu;
        const long long pr = pair0 + t;
        if (pr >= npairs) continue;
        const long long cw = pr / VP;
        const int v = (int)(pr % VP) * 2;
        const C zk = res[k * ld + t];
        const C zm = res[((P - k) % P) * ld + t];
        C A, B;
        A.x = (R)0.5 * (zk.x + zm.x);
        A.y = (R)0.5 * (zk.y - zm.y);
        B.x = (R)0.5 * (zk.y + zm.y);
        B.y = (R)0.5 * (zm.x - zk.x);
        out[(cw * V + v) * (long long)Hu + k] = A;
        if (v + 1 < V) out[(cw * V + v + 1) * (long long)Hu + k] = B;
    }
}

// ------------------------------------------------------------------ pass x, inverse
// [3][W][V][Hu] Hermitian halves -> real rows [3][W][V][U] (first U outputs)
template <typename R>
__global__ void __launch_bounds__(NT) k_inv_x(const typename CT<R>::c* __restrict__ in, int U,
                                              int V, int W, R* __restrict__ out,
                                              const typename CT<R>::c* __restrict__ tw,
                                              RadixList rl) {
    typedef typename CT<R>::c C;
    constexpr int TB = Tile<R>::TB;
    constexpr int ld = TB + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* stw = reinterpret_cast<C*>(smem_raw);
    C* b0 = stw + tw_entries<C>(rl.P);
    C* b1 = b0 + rl.P * ld;
    const int P = rl.P, Hu = P / 2 + 1;
    const int VP = (V + 1) / 2;
    const long long npairs = 3LL * W * VP;
    const long long pair0 = (long long)blockIdx.x * TB;
    load_tw(stw, tw, P);
    for (int it0 = threadIdx.x; it0 < TB * Hu; it0 += kLoadBatch * blockDim.x) {
        C Aq[kLoadBatch], Bq[kLoadBatch];
#pragma unroll
        for (int q = 0; q < kLoadBatch; ++q) {
            const int it = it0 + q * blockDim.x;
            const int t = it / Hu, k = it % Hu;
            const long long pr = pair0 + t;
            Aq[q].x = 0; Aq[q].y = 0; Bq[q].x = 0; Bq[q].y = 0;
            if (it < TB * Hu && pr < npairs) {
                const long long cw = pr / VP;
                const int v = (int)(pr % VP) * 2;
                Aq[q] = in[(cw * V + v) * (long long)Hu + k];
                if (v + 1 < V) Bq[q] = in[(cw * V + v + 1) * (long long)Hu + k];
            }
        }
#pragma unroll
        for (int q = 0; q < kLoadBatch; ++q) {
            const int it = it0 + q * blockDim.x;
            if (it >= TB * Hu) break;
            const int t = it / Hu, k = it % Hu;
            const C A = Aq[q], B = Bq[q];
            C z;
            z.x = A.x - B.y;
            z.y = A.y + B.x;
            b0[k * ld + t] = z;
            if (k >= 1 && k < P - k) {
                C zm;
                zm.x = A.x + B.y;
                zm.y = B.x - A.y;
                b0[(P - k) * ld + t] = zm;
            }
        }
    }
    __syncthreads();
    C* res = fft_tile<C, TB>(b0, b1, P, rl.r, rl.n, ld, stw, +1);
    for (int it = threadIdx.x; it < TB * U; it += blockDim.x) {
        const int t = it / U, j = it % U;
        const long long pr = pair0 + t;
        if (pr >= npairs) continue;
        const long long cw = pr / VP;
        const int v = (int)(pr % VP) * 2;
        const C z = res[j * ld + t];
        out[(cw * V + v) * (long long)U + j] = z.x;
        if (v + 1 < V) out[(cw * V + v + 1) * (long long)U + j] = z.y;
    }
}

// ------------------------------------------------------------------ pass x, four-step codelets
// For P = P1 P2 (64 = 8 x 8, 96 = 8 x 12, 210 = 14 x 15): 32 row pairs per CTA, each
// pair a complex line of P points in shared memory ([P][33], line fastest).  Phase A
// (warp n1 < P1, lane = line): x[n1 + P1 n2] -> DFT of length P2 over n2 in registers
// (compile-time radices and twiddles, dft_ct) -> times W_P^{n1 k2}; phase B (warp
// k2 < P2): DFT of length P1 over n1 -> X[k2 + P2 k1].  Every phase first reads its
// values into registers, then (after a barrier) writes them back into the same buffer.
constexpr int kXL = 32;          // row pairs per CTA
constexpr int kXLD = kXL + 1;    // padded line stride of the shared buffer

template <typename C, int P1, int P2, int DIR>
__device__ __forceinline__ void x_four_step(C* X, const C* stw, int nvalid) {
    constexpr int P = P1 * P2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    C x[P2];
    if (warp < P1) {
        const int n1 = warp;
        Unroll1<0, P2>::run([&](auto q) {
            constexpr int n2 = decltype(q)::value;
            const int idx = n1 + P1 * n2;
            C v;
            v.x = 0; v.y = 0;
            if (idx < nvalid) v = X[idx * kXLD + lane];
            x[n2] = v;
        });
        dft_ct<P2, DIR>(x);
        Unroll1<0, P2>::run([&](auto q) {
            constexpr int k2 = decltype(q)::value;
            x[k2] = twmul_tab(stw, (n1 * k2) % P, P, DIR, x[k2]);
        });
    }
    __syncthreads();
    if (warp < P1)
        Unroll1<0, P2>::run([&](auto q) {
            constexpr int k2 = decltype(q)::value;
            X[(warp * P2 + k2) * kXLD + lane] = x[k2];
        });
    __syncthreads();
    C y[P1];
    if (warp < P2) {
        Unroll1<0, P1>::run([&](auto q) {
            constexpr int n1 = decltype(q)::value;
            y[n1] = X[(n1 * P2 + warp) * kXLD + lane];
        });
        dft_ct<P1, DIR>(y);
    }
    __syncthreads();
    if (warp < P2)
        Unroll1<0, P1>::run([&](auto q) {
            constexpr int k1 = decltype(q)::value;
            X[(warp + P2 * k1) * kXLD + lane] = y[k1];
        });
    __syncthreads();
}

template <typename R, int P1, int P2>
__global__ void k_fwd_x4s(const double* __restrict__ in, int U, int V, int W,
                          typename CT<R>::c* __restrict__ out,
                          const typename CT<R>::c* __restrict__ tw,
                          const double* __restrict__ scale) {
    typedef typename CT<R>::c C;
    constexpr int P = P1 * P2, Hu = P / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* X = reinterpret_cast<C*>(smem_raw);          // [P][kXLD]
    C* stw = X + P * kXLD;                          // [tw_entries(P)]
    const int VP = (V + 1) / 2;
    const long long npairs = 3LL * W * VP;
    const long long pair0 = (long long)blockIdx.x * kXL;
    for (int i = threadIdx.x; i < tw_entries<C>(P); i += blockDim.x) stw[i] = tw[i];
    // z = a + i b of the two rows of a pair; positions >= U are the zero padding
    for (int it = threadIdx.x; it < kXL * U; it += blockDim.x) {
        const int t = it / U, j = it % U;
        const long long pr = pair0 + t;
        double va = 0.0, vb = 0.0;
        if (pr < npairs) {
            const long long cw = pr / VP;
            const int v = (int)(pr % VP) * 2;
            const double* row = in + (cw * V + v) * (long long)U;
            va = row[j];
            if (v + 1 < V) vb = row[U + j];
            if (scale) {   // per-voxel factor (the adjoint transforms chi * lambda)
                const long long m0 = ((cw % W) * V + v) * (long long)U + j;
                va *= scale[m0];
                if (v + 1 < V) vb *= scale[m0 + U];
            }
        }
        C z;
        z.x = (R)va;
        z.y = (R)vb;
        X[j * kXLD + t] = z;
    }
    __syncthreads();
    x_four_step<C, P1, P2, -1>(X, stw, U);
    // split: A = (Z[k] + conj Z[P-k]) / 2, B = -i (Z[k] - conj Z[P-k]) / 2
    for (int it = threadIdx.x; it < kXL * Hu; it += blockDim.x) {
        const int t = it / Hu, k = it % Hu;
        const long long pr = pair0 + t;
        if (pr >= npairs) continue;
        const long long cw = pr / VP;
        const int v = (int)(pr % VP) * 2;
        const C zk = X[k * kXLD + t];
        const C zm = X[((P - k) % P) * kXLD + t];
        C A, B;
        A.x = (R)0.5 * (zk.x + zm.x);
        A.y = (R)0.5 * (zk.y - zm.y);
        B.x = (R)0.5 * (zk.y + zm.y);
        B.y = (R)0.5 * (zm.x - zk.x);
        out[(cw * V + v) * (long long)Hu + k] = A;
        if (v + 1 < V) out[(cw * V + v + 1) * (long long)Hu + k] = B;
    }
}

template <typename R, int P1, int P2>
__global__ void k_inv_x4s(const typename CT<R>::c* __restrict__ in, int U, int V, int W,
                          R* __restrict__ out, const typename CT<R>::c* __restrict__ tw) {
    typedef typename CT<R>::c C;
    constexpr int P = P1 * P2, Hu = P / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* X = reinterpret_cast<C*>(smem_raw);
    C* stw = X + P * kXLD;
    const int VP = (V + 1) / 2;
    const long long npairs = 3LL * W * VP;
    const long long pair0 = (long long)blockIdx.x * kXL;
    for (int i = threadIdx.x; i < tw_entries<C>(P); i += blockDim.x) stw[i] = tw[i];
    // Z[k] = A[k] + i B[k] and Z[P-k] = conj A[k] + i conj B[k] from the two halves
    for (int it = threadIdx.x; it < kXL * Hu; it += blockDim.x) {
        const int t = it / Hu, k = it % Hu;
        const long long pr = pair0 + t;
        C A, B;
        A.x = 0; A.y = 0; B.x = 0; B.y = 0;
        if (pr < npairs) {
            const long long cw = pr / VP;
            const int v = (int)(pr % VP) * 2;
            A = in[(cw * V + v) * (long long)Hu + k];
            if (v + 1 < V) B = in[(cw * V + v + 1) * (long long)Hu + k];
        }
        C z;
        z.x = A.x - B.y;
        z.y = A.y + B.x;
        X[k * kXLD + t] = z;
        if (k >= 1 && k < P - k) {
            C zm;
            zm.x = A.x + B.y;
            zm.y = B.x - A.y;
            X[(P - k) * kXLD + t] = zm;
        }
    }
    __syncthreads();
    x_four_step<C, P1, P2, +1>(X, stw, P);
    for (int it = threadIdx.x; it < kXL * U; it += blockDim.x) {
        const int t = it / U, j = it % U;
        const long long pr = pair0 + t;
        if (pr >= npairs) continue;
        const long long cw = pr / VP;
        const int v = (int)(pr % VP) * 2;
        const C z = X[j * kXLD + t];
        out[(cw * V + v) * (long long)U + j] = z.x;
        if (v + 1 < V) out[(cw * V + v + 1) * (long long)U + j] = z.y;
    }
}

// ------------------------------------------------------------------ strided passes
struct MidArgs {
    int n_in, n_out;          // inputs read / outputs stored along the axis
    int n_o2;                 // outer index o = comp * n_o2 + o2
    long long in_c, in_o, in_a;    // strides: component, outer, axis (in elements)
    long long out_c, out_o, out_a;
    int Hu;                   // contiguous extent tiled by TB
    int dir;
};

template <typename R>
__global__ void __launch_bounds__(NT) k_mid(const typename CT<R>::c* __restrict__ in,
                                            typename CT<R>::c* __restrict__ out,
                                            const typename CT<R>::c* __restrict__ tw,
                                            RadixList rl, MidArgs a) {
    typedef typename CT<R>::c C;
    constexpr int TB = Tile<R>::TB;
    constexpr int ld = TB + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* stw = reinterpret_cast<C*>(smem_raw);
    C* b0 = stw + tw_entries<C>(rl.P);
    C* b1 = b0 + rl.P * ld;
    const int P = rl.P;
    const int ntile = (a.Hu + TB - 1) / TB;
    const long long o = blockIdx.x / ntile;
    const int ku0 = (int)(blockIdx.x % ntile) * TB;
    const long long comp = o / a.n_o2, o2 = o % a.n_o2;
    const C* src = in + comp * a.in_c + o2 * a.in_o + ku0;
    C* dst = out + comp * a.out_c + o2 * a.out_o + ku0;
    load_tw(stw, tw, P);
    for (int it = threadIdx.x; it < P * TB; it += blockDim.x) {
        const int j = it / TB, t = it % TB;
        const bool ok = j < a.n_in && ku0 + t < a.Hu;
        cp_async_c(&b0[j * ld + t], ok ? src + j * a.in_a + t : src, ok);
    }
    cp_async_commit_wait();
    __syncthreads();
    C* res = fft_tile<C, TB>(b0, b1, P, rl.r, rl.n, ld, stw, a.dir);
    for (int it = threadIdx.x; it < a.n_out * TB; it += blockDim.x) {
        const int j = it / TB, t = it % TB;
        if (ku0 + t < a.Hu) dst[j * a.out_a + t] = res[j * ld + t];
    }
}

// ------------------------------------------------------------------ strided passes, four-step
// Length P = P1 P2 with both factors small: n = n1 + P1 n2, k = k2 + P2 k1,
//   X[k2 + P2 k1] = sum_{n1} W_P1^{n1 k1} (W_P^{n1 k2} sum_{n2} x[n1 + P1 n2] W_P2^{n2 k2}).
// A CTA holds 32 consecutive lines (lane = line, so every load and store is one
// coalesced run); phase A: warp n1 loads its P2 strided inputs (only the unpadded
// ones), runs the P2-point DFT in registers (compile-time structure and roots) and
// applies W_P^{n1 k2}; phase B: warp k2 gathers the P1 values over n1 from shared
// memory, runs the P1-point DFT and stores the outputs the pass needs.
template <typename R, int P1, int P2, int DIR>
__global__ void __launch_bounds__(32 * (P1 > P2 ? P1 : P2))
k_mid4s(const typename CT<R>::c* __restrict__ in, typename CT<R>::c* __restrict__ out,
        const typename CT<R>::c* __restrict__ tw, MidArgs a) {
    typedef typename CT<R>::c C;
    constexpr int P = P1 * P2, NL = 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Y = reinterpret_cast<C*>(smem_raw);          // [P1][P2][NL]
    C* stw = Y + P * NL;                            // roots exp(-2 pi i k / P) (tw_entries)
    const int ntile = (a.Hu + NL - 1) / NL;
    const long long o = blockIdx.x / ntile;
    const int ku0 = (int)(blockIdx.x % ntile) * NL;
    const long long comp = o / a.n_o2, o2 = o % a.n_o2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool live = ku0 + lane < a.Hu;
    const C* src = in + comp * a.in_c + o2 * a.in_o + ku0 + lane;
    C* dst = out + comp * a.out_c + o2 * a.out_o + ku0 + lane;
    for (int i = threadIdx.x; i < tw_entries<C>(P); i += blockDim.x) stw[i] = tw[i];
    __syncthreads();
    if (warp < P1) {
        const int n1 = warp;
        C x[P2];
        Unroll1<0, P2>::run([&](auto q) {
            constexpr int n2 = decltype(q)::value;
            const int idx = n1 + P1 * n2;
            C v;
            v.x = 0; v.y = 0;
            if (idx < a.n_in && live) v = src[(long long)idx * a.in_a];
            x[n2] = v;
        });
        dft_ct<P2, DIR>(x);
        Unroll1<0, P2>::run([&](auto q) {
            constexpr int k2 = decltype(q)::value;
            Y[(n1 * P2 + k2) * NL + lane] = twmul_tab(stw, (n1 * k2) % P, P, DIR, x[k2]);
        });
    }
    __syncthreads();
    if (warp < P2) {
        const int k2 = warp;
        C y[P1];
        Unroll1<0, P1>::run([&](auto q) {
            constexpr int n1 = decltype(q)::value;
            y[n1] = Y[(n1 * P2 + k2) * NL + lane];
        });
        dft_ct<P1, DIR>(y);
        if (!live) return;
        Unroll1<0, P1>::run([&](auto q) {
            constexpr int k1 = decltype(q)::value;
            const int k = k2 + P2 * k1;
            if (k < a.n_out) dst[(long long)k * a.out_a] = y[k1];
        });
    }
}

RadixList radix_list(const AxisFFT& ax) {
    RadixList rl;
    rl.P = ax.P;
    rl.n = ax.nrad;
    for (int i = 0; i < 16; ++i) rl.r[i] = ax.rad[i];
    return rl;
}

template <typename R> const typename CT<R>::c* table(const AxisFFT& a);
template <> const double2* table<double>(const AxisFFT& a) { return a.tw64; }
template <> const float2* table<float>(const AxisFFT& a) { return a.tw32; }

template <typename R> size_t smem_bytes(int P) {
    typedef typename CT<R>::c C;
    return sizeof(C) * ((size_t)tw_entries<C>(P) + 2 * (size_t)P * (Tile<R>::TB + 1));
}

// Dynamic shared memory of a pass kernel.  The limit is a process-wide attribute of
// the kernel, and contexts of different sizes may launch it from several threads, so
// it is set to the device's opt-in maximum (a value that never changes) rather than
// to one launch's need; the need is checked against it.  The largest shared-memory
// carveout is preferred so that several tiles are resident per SM.
template <typename K> void set_smem(K kern, size_t bytes) {
    int dev = 0, optin = 0;
    MOT_CUDA_TRY(cudaGetDevice(&dev));
    MOT_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (bytes > (size_t)optin)
        throw MotError{MOT_ERR_ARG, "FFT length too large for one shared-memory tile"};
    MOT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    MOT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
}

template <typename R, int P1, int P2>
void launch_mid4s(const typename CT<R>::c* in, typename CT<R>::c* out,
                  const typename CT<R>::c* tw, const MidArgs& a, int nblocks, cudaStream_t s) {
    typedef typename CT<R>::c C;
    const size_t sm = sizeof(C) * ((size_t)P1 * P2 * 32 + (size_t)tw_entries<C>(P1 * P2));
    constexpr int threads = 32 * (P1 > P2 ? P1 : P2);
    if (a.dir < 0) {
        set_smem(k_mid4s<R, P1, P2, -1>, sm);
        k_mid4s<R, P1, P2, -1><<<nblocks, threads, sm, s>>>(in, out, tw, a);
    } else {
        set_smem(k_mid4s<R, P1, P2, +1>, sm);
        k_mid4s<R, P1, P2, +1><<<nblocks, threads, sm, s>>>(in, out, tw, a);
    }
    MOT_LAUNCH_CHECK();
}

// a strided pass of length ax.P over [3][n_o2] x Hu lines: the four-step kernel for the
// lengths that have a factor pair below, the generic Stockham tile otherwise
template <typename R>
void mid_pass(const typename CT<R>::c* in, typename CT<R>::c* out, const AxisFFT& ax,
              const MidArgs& a, cudaStream_t s) {
    const int P = ax.P;
    const long long lines = 3LL * a.n_o2;
    const int nb32 = (int)(lines * ((a.Hu + 31) / 32));
    switch (P) {
        case 64: launch_mid4s<R, 8, 8>(in, out, table<R>(ax), a, nb32, s); return;
        case 96: launch_mid4s<R, 8, 12>(in, out, table<R>(ax), a, nb32, s); return;
        case 210: launch_mid4s<R, 14, 15>(in, out, table<R>(ax), a, nb32, s); return;
        default: break;
    }
    constexpr int TB = Tile<R>::TB;
    const size_t sm = smem_bytes<R>(P);
    set_smem(k_mid<R>, sm);
    k_mid<R><<<(int)(lines * ((a.Hu + TB - 1) / TB)), NT, sm, s>>>(in, out, table<R>(ax),
                                                                    radix_list(ax), a);
    MOT_LAUNCH_CHECK();
}

__global__ void twiddle_kernel(int P, double2* t64, float2* t32) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)P, &s, &c);
    t64[k] = make_double2(c, -s);
    const float2 h = make_float2((float)c, (float)-s);
    t32[k] = h;                                                   // hi
    t32[P + k] = make_float2((float)(c - (double)h.x), (float)(-s - (double)h.y));   // lo
}

}  // namespace

namespace mot {

void fft_plan_axis(AxisFFT& a, int P) {
    a.P = P;
    a.nrad = 0;
    int n = P;
    while (n % 4 == 0) { a.rad[a.nrad++] = 4; n /= 4; }
    while (n % 2 == 0) { a.rad[a.nrad++] = 2; n /= 2; }
    for (int r : {3, 5, 7})
        while (n % r == 0) { a.rad[a.nrad++] = r; n /= r; }
    if (n != 1) throw MotError{MOT_ERR_ARG, "FFT length has a prime factor above 7"};
    MOT_CUDA_TRY(cudaMalloc(&a.tw64, sizeof(double2) * P));
    MOT_CUDA_TRY(cudaMalloc(&a.tw32, sizeof(float2) * 2 * P));
    twiddle_kernel<<<(P + 255) / 256, 256>>>(P, a.tw64, a.tw32);
    MOT_LAUNCH_CHECK();
    MOT_CUDA_TRY(cudaDeviceSynchronize());
}

void fft_free_axis(AxisFFT& a) {
    cudaFree(a.tw64);
    cudaFree(a.tw32);
    a.tw64 = nullptr;
    a.tw32 = nullptr;
}

// x passes through the four-step codelets where P has one (false: use the generic kernel)
template <typename R, int P1, int P2>
void launch_x4s(bool fwd, mot_ctx* c, const double* Jsoa, typename CT<R>::c* spec, R* real,
                const double* scale, cudaStream_t s) {
    typedef typename CT<R>::c C;
    constexpr int P = P1 * P2;
    const size_t sm = sizeof(C) * ((size_t)P * kXLD + tw_entries<C>(P));
    const int threads = 32 * (P1 > P2 ? P1 : P2);
    const long long npairs = 3LL * c->W * ((c->V + 1) / 2);
    const int blocks = (int)((npairs + kXL - 1) / kXL);
    if (fwd) {
        set_smem(k_fwd_x4s<R, P1, P2>, sm);
        k_fwd_x4s<R, P1, P2><<<blocks, threads, sm, s>>>(Jsoa, c->U, c->V, c->W, spec,
                                                         table<R>(c->ax[0]), scale);
    } else {
        set_smem(k_inv_x4s<R, P1, P2>, sm);
        k_inv_x4s<R, P1, P2><<<blocks, threads, sm, s>>>(spec, c->U, c->V, c->W, real,
                                                         table<R>(c->ax[0]));
    }
    MOT_LAUNCH_CHECK();
}

template <typename R>
bool x_pass_codelet(bool fwd, mot_ctx* c, const double* Jsoa, typename CT<R>::c* spec, R* real,
                    const double* scale, cudaStream_t s) {
    switch (c->ax[0].P) {
        case 64: launch_x4s<R, 8, 8>(fwd, c, Jsoa, spec, real, scale, s); return true;
        case 96: launch_x4s<R, 8, 12>(fwd, c, Jsoa, spec, real, scale, s); return true;
        case 210: launch_x4s<R, 14, 15>(fwd, c, Jsoa, spec, real, scale, s); return true;
        default: return false;
    }
}

template <typename R>
void fft_forward(mot_ctx* c, const double* Jsoa, typename CT<R>::c* out, cudaStream_t s,
                 const double* scale) {
    typedef typename CT<R>::c C;
    HistoryBuffers<R>& hb = hbuf<R>(c);
    constexpr int TB = Tile<R>::TB;
    const int U = c->U, V = c->V, W = c->W;
    const int Pu = c->ax[0].P, Pv = c->ax[1].P, Pw = c->ax[2].P, Hu = c->Hu;
    // x
    if (!x_pass_codelet<R>(true, c, Jsoa, hb.tmp1, nullptr, scale, s)) {
        const long long npairs = 3LL * W * ((V + 1) / 2);
        const size_t sm = smem_bytes<R>(Pu);
        set_smem(k_fwd_x<R>, sm);
        k_fwd_x<R><<<(int)((npairs + TB - 1) / TB), NT, sm, s>>>(Jsoa, U, V, W, hb.tmp1,
                                                                 table<R>(c->ax[0]),
                                                                 radix_list(c->ax[0]), scale);
        MOT_LAUNCH_CHECK();
    }
    // y: [3][W][V][Hu] -> [3][W][Pv][Hu]
    {
        MidArgs a;
        a.n_in = V; a.n_out = Pv; a.n_o2 = W;
        a.in_c = (long long)W * V * Hu; a.in_o = (long long)V * Hu; a.in_a = Hu;
        a.out_c = (long long)W * Pv * Hu; a.out_o = (long long)Pv * Hu; a.out_a = Hu;
        a.Hu = Hu; a.dir = -1;
        mid_pass<R>(hb.tmp1, hb.tmp2, c->ax[1], a, s);
    }
    // z: [3][W][Pv][Hu] -> [3][Pw][Pv][Hu]
    {
        MidArgs a;
        a.n_in = W; a.n_out = Pw; a.n_o2 = Pv;
        a.in_c = (long long)W * Pv * Hu; a.in_o = Hu; a.in_a = (long long)Pv * Hu;
        a.out_c = (long long)Pw * Pv * Hu; a.out_o = Hu; a.out_a = (long long)Pv * Hu;
        a.Hu = Hu; a.dir = -1;
        mid_pass<R>(hb.tmp2, out, c->ax[2], a, s);
    }
}

template <typename R>
void fft_inverse(mot_ctx* c, const typename CT<R>::c* in, R* out, cudaStream_t s) {
    HistoryBuffers<R>& hb = hbuf<R>(c);
    constexpr int TB = Tile<R>::TB;
    const int U = c->U, V = c->V, W = c->W;
    const int Pu = c->ax[0].P, Pv = c->ax[1].P, Pw = c->ax[2].P, Hu = c->Hu;
    // z: [3][Pw][Pv][Hu] -> [3][W][Pv][Hu]
    {
        MidArgs a;
        a.n_in = Pw; a.n_out = W; a.n_o2 = Pv;
        a.in_c = (long long)Pw * Pv * Hu; a.in_o = Hu; a.in_a = (long long)Pv * Hu;
        a.out_c = (long long)W * Pv * Hu; a.out_o = Hu; a.out_a = (long long)Pv * Hu;
        a.Hu = Hu; a.dir = +1;
        mid_pass<R>(in, hb.tmp2, c->ax[2], a, s);
    }
    // y: [3][W][Pv][Hu] -> [3][W][V][Hu]
    {
        MidArgs a;
        a.n_in = Pv; a.n_out = V; a.n_o2 = W;
        a.in_c = (long long)W * Pv * Hu; a.in_o = (long long)Pv * Hu; a.in_a = Hu;
        a.out_c = (long long)W * V * Hu; a.out_o = (long long)V * Hu; a.out_a = Hu;
        a.Hu = Hu; a.dir = +1;
        mid_pass<R>(hb.tmp2, hb.tmp1, c->ax[1], a, s);
    }
    // x: c2r
    if (!x_pass_codelet<R>(false, c, nullptr, hb.tmp1, out, nullptr, s)) {
        const long long npairs = 3LL * W * ((V + 1) / 2);
        const size_t sm = smem_bytes<R>(Pu);
        set_smem(k_inv_x<R>, sm);
        k_inv_x<R><<<(int)((npairs + TB - 1) / TB), NT, sm, s>>>(hb.tmp1, U, V, W, out,
                                                                 table<R>(c->ax[0]),
                                                                 radix_list(c->ax[0]));
        MOT_LAUNCH_CHECK();
    }
}

template void fft_forward<double>(mot_ctx*, const double*, double2*, cudaStream_t, const double*);
template void fft_forward<float>(mot_ctx*, const double*, float2*, cudaStream_t, const double*);
template void fft_inverse<double>(mot_ctx*, const double2*, double*, cudaStream_t);
template void fft_inverse<float>(mot_ctx*, const float2*, float*, cudaStream_t);

}  // namespace mot

// Scattered field at probe voxels and its transpose: the objective of the adjoint
// workload (time-gated field energy at probes around the scatterer) on the device.
//
// A probe is a voxel of the grid's lattice (inside or outside the grid); its field is
// the tested (voxel-averaged) field of Eq. E at that virtual vacuum voxel, which the
// march's own elements give (Eq. Z, no local term in vacuum):
//     E^s_p(t_n) = sum_{l>=0} sum_m G_l(r_p - r_m) J_{n-l,m},
// and the transposed operator, the source of the adjoint march for an objective of E^s,
//     g_{k,m} = sum_{l>=0} sum_p G_l(r_p - r_m)^T W_{k+l,p}         (G_l^T = G_l).
// The elements of every probe-voxel pair are windows of WIN lags from the element
// quadrature (mot_probe_setup); both products run in FP64 with one thread per voxel
// and a block of time steps per thread.
#include "mot_internal.cuh"

#include <algorithm>
#include <new>
#include <vector>

namespace {

constexpr int PT = 256;    // threads per block
constexpr int TBN = 8;     // time steps per block

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// E[n][p][a], n in [n0, n0 + TBN): one block per (time block, probe), threads over the
// voxels; every thread keeps the partial sums of its voxels, reduced over the block
__global__ void __launch_bounds__(PT) k_probe_field(const double* __restrict__ tab,
                                                    const int* __restrict__ l0, long long M,
                                                    int N, int P, const double* __restrict__ J,
                                                    double* __restrict__ E) {
    const int p = blockIdx.y;
    const int n0 = blockIdx.x * TBN;
    double acc[TBN][3];
#pragma unroll
    for (int k = 0; k < TBN; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.0;
    const double* tp = tab + (long long)p * 6 * mot::WIN * M;
    for (long long m = threadIdx.x; m < M; m += PT) {
        const int lo = l0[(long long)p * M + m];
#pragma unroll
        for (int i = 0; i < mot::WIN; ++i) {
            const double gxx = tp[(0 * mot::WIN + i) * M + m], gyy = tp[(1 * mot::WIN + i) * M + m];
            const double gzz = tp[(2 * mot::WIN + i) * M + m], gxy = tp[(3 * mot::WIN + i) * M + m];
            const double gxz = tp[(4 * mot::WIN + i) * M + m], gyz = tp[(5 * mot::WIN + i) * M + m];
#pragma unroll
            for (int k = 0; k < TBN; ++k) {
                const int n = n0 + k - lo - i;           // J index of J_{n-l}, 0-based
                if (n < 0 || n0 + k >= N) continue;
                const double* j = J + ((long long)n * M + m) * 3;
                const double j0 = j[0], j1 = j[1], j2 = j[2];
                acc[k][0] += gxx * j0 + gxy * j1 + gxz * j2;
                acc[k][1] += gxy * j0 + gyy * j1 + gyz * j2;
                acc[k][2] += gxz * j0 + gyz * j1 + gzz * j2;
            }
        }
    }
    // block reduction of the TBN x 3 sums: warp shuffles, then one value per warp
    __shared__ double red[PT / 32][TBN * 3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < TBN; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = acc[k][a];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][k * 3 + a] = v;
        }
    __syncthreads();
    if (threadIdx.x < TBN * 3) {
        const int k = threadIdx.x / 3, a = threadIdx.x % 3;
        double s = 0.0;
        for (int w = 0; w < PT / 32; ++w) s += red[w][threadIdx.x];
        if (n0 + k < N) E[((long long)(n0 + k) * P + p) * 3 + a] = s;
    }
}

// g[k][m][b] for k in [k0, k0 + TBN): one thread per voxel, probes in turn
__global__ void __launch_bounds__(PT) k_probe_transpose(const double* __restrict__ tab,
                                                        const int* __restrict__ l0, long long M,
                                                        int N, int P, const double* __restrict__ W,
                                                        double* __restrict__ g) {
    const long long m = (long long)blockIdx.x * PT + threadIdx.x;
    const int k0 = blockIdx.y * TBN;
    if (m >= M) return;
    double acc[TBN][3];
#pragma unroll
    for (int k = 0; k < TBN; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.0;
    for (int p = 0; p < P; ++p) {
        const double* tp = tab + (long long)p * 6 * mot::WIN * M;
        const int lo = l0[(long long)p * M + m];
#pragma unroll
        for (int i = 0; i < mot::WIN; ++i) {
            const double gxx = tp[(0 * mot::WIN + i) * M + m], gyy = tp[(1 * mot::WIN + i) * M + m];
            const double gzz = tp[(2 * mot::WIN + i) * M + m], gxy = tp[(3 * mot::WIN + i) * M + m];
            const double gxz = tp[(4 * mot::WIN + i) * M + m], gyz = tp[(5 * mot::WIN + i) * M + m];
#pragma unroll
            for (int k = 0; k < TBN; ++k) {
                const int n = k0 + k + lo + i;           // field time of W_{k+l}, 0-based
                if (n >= N) continue;
                const double* w = W + ((long long)n * P + p) * 3;
                const double w0 = w[0], w1 = w[1], w2 = w[2];
                acc[k][0] += gxx * w0 + gxy * w1 + gxz * w2;
                acc[k][1] += gxy * w0 + gyy * w1 + gyz * w2;
                acc[k][2] += gxz * w0 + gyz * w1 + gzz * w2;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < TBN; ++k) {
        if (k0 + k >= N) break;
        double* dst = g + ((long long)(k0 + k) * M + m) * 3;
        dst[0] = acc[k][0];
        dst[1] = acc[k][1];
        dst[2] = acc[k][2];
    }
}

template <typename F>
mot_status guarded_probe(mot_ctx* c, F&& f) {
    if (c->broken) return MOT_ERR_STATE;
    try {
        f();
        return MOT_OK;
    } catch (const MotError& e) {
        c->err = e.msg;
        if (e.st == MOT_ERR_CUDA || e.st == MOT_ERR_TIMEOUT) c->broken = true;
        return e.st;
    } catch (const std::bad_alloc&) {
        c->err = "host allocation failed";
        return MOT_ERR_OOM;
    }
}

// device view of a caller buffer of `count` doubles: itself, or a staged copy
const double* stage_in(const double* src, long long count, std::vector<void*>& owned,
                       cudaStream_t s) {
    if (on_device(src)) return src;
    double* d = nullptr;
    MOT_CUDA_TRY(cudaMalloc(&d, sizeof(double) * count));
    owned.push_back(d);
    MOT_CUDA_TRY(cudaMemcpyAsync(d, src, sizeof(double) * count, cudaMemcpyHostToDevice, s));
    return d;
}

}  // namespace

extern "C" {

mot_status mot_probe_setup(mot_ctx* c, int n_probes, const int* probes) {
    if (!c) return MOT_ERR_ARG;
    if (n_probes < 1 || !probes) {
        c->err = "mot_probe_setup needs n_probes >= 1 and a host array of [n][3] indices";
        return MOT_ERR_ARG;
    }
    return guarded_probe(c, [&] {
        cudaFree(c->probe_tab);
        cudaFree(c->probe_l0);
        c->probe_tab = nullptr;
        c->probe_l0 = nullptr;
        c->n_probes = 0;
        MOT_CUDA_TRY(cudaMalloc(&c->probe_tab, sizeof(double) * (size_t)n_probes * 6 * mot::WIN * c->M));
        MOT_CUDA_TRY(cudaMalloc(&c->probe_l0, sizeof(int) * (size_t)n_probes * c->M));
        mot::probe_windows(c, n_probes, probes, c->probe_tab, c->probe_l0);
        c->n_probes = n_probes;
    });
}

mot_status mot_probe_field(mot_ctx* c, int n_steps, const double* J, double* E, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (!c->n_probes) { c->err = "no probes (mot_probe_setup first)"; return MOT_ERR_ARG; }
    if (n_steps < 1 || !J || !E) { c->err = "n_steps >= 1 and non-null buffers required"; return MOT_ERR_ARG; }
    std::vector<void*> owned;
    mot_status st = guarded_probe(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        const double* Jd = stage_in(J, 3LL * c->M * n_steps, owned, s);
        const long long ne = 3LL * c->n_probes * n_steps;
        double* Ed = E;
        const bool host_out = !on_device(E);
        if (host_out) {
            MOT_CUDA_TRY(cudaMalloc(&Ed, sizeof(double) * ne));
            owned.push_back(Ed);
        }
        dim3 grid((n_steps + TBN - 1) / TBN, c->n_probes);
        k_probe_field<<<grid, PT, 0, s>>>(c->probe_tab, c->probe_l0, c->M, n_steps, c->n_probes, Jd,
                                          Ed);
        MOT_LAUNCH_CHECK();
        if (host_out)
            MOT_CUDA_TRY(cudaMemcpyAsync(E, Ed, sizeof(double) * ne, cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
    });
    for (void* p : owned) cudaFree(p);
    return st;
}

mot_status mot_probe_transpose(mot_ctx* c, int n_steps, const double* W, double* g, void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (!c->n_probes) { c->err = "no probes (mot_probe_setup first)"; return MOT_ERR_ARG; }
    if (n_steps < 1 || !W || !g) { c->err = "n_steps >= 1 and non-null buffers required"; return MOT_ERR_ARG; }
    std::vector<void*> owned;
    mot_status st = guarded_probe(c, [&] {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        const double* Wd = stage_in(W, 3LL * c->n_probes * n_steps, owned, s);
        const long long ng = 3LL * c->M * n_steps;
        double* gd = g;
        const bool host_out = !on_device(g);
        if (host_out) {
            MOT_CUDA_TRY(cudaMalloc(&gd, sizeof(double) * ng));
            owned.push_back(gd);
        }
        dim3 grid((unsigned)((c->M + PT - 1) / PT), (n_steps + TBN - 1) / TBN);
        k_probe_transpose<<<grid, PT, 0, s>>>(c->probe_tab, c->probe_l0, c->M, n_steps,
                                              c->n_probes, Wd, gd);
        MOT_LAUNCH_CHECK();
        if (host_out)
            MOT_CUDA_TRY(cudaMemcpyAsync(g, gd, sizeof(double) * ng, cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
    });
    for (void* p : owned) cudaFree(p);
    return st;
}

}  // extern "C"

// Per-step right-hand side (FIR epilogue) and near-field solve (Eq. MOTInversion).
//
//   rhs_m  = E_{n,m} - P_{n-1,m},
//   P_{n-1,m} = T(1)/eps_m J_{n-1,m} + sum_{l=1}^{L-1} delta_l J_{n-l,m} - chi_m (G * J)_hist,m
// with T(1) = 1/2 (Sec. 2.3 reading) and the FIR taps delta_l of Sec. 6.1.
//
// Z_0^delta = diag(T(0)/eps + delta_0) - diag(chi) G_0 couples each voxel to its 26
// neighbours when c dt = h (Sec. 5.2).  Scaled by diag(1/chi) it is symmetric positive
// definite on the voxels with chi > 0 (D_0 = Z_0 in the PDSA, Eq. Dn), so it is solved
// with conjugate gradients on A = diag((T(0)/eps + delta_0)/chi) - G_0 and b = rhs/chi.
// Voxels with eps = 1 (chi = 0) carry J = rhs / (T(0) + delta_0), which is zero for
// the zero initial state.  The CG runs as one cooperative kernel with grid-wide
// barriers; it stops at ||r|| <= tol ||b|| or after max_iter iterations.
#include "mot_internal.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace {

constexpr int NT = 256;
constexpr int MAXTAPS = 64;

__constant__ double c_stencil[27 * 6];   // G_0(e) for e in {-1,0,1}^3, order xx yy zz xy xz yz
__constant__ double c_taps[MAXTAPS];

// ring slot of J_{n-l}: (s0 - l) mod jring, s0 = n mod jring, 0 <= l < jring
__device__ __forceinline__ long long jslot(int s0, int l, int jring, long long stride) {
    int sl = s0 - l;
    if (sl < 0) sl += jring;
    return (long long)sl * stride;
}

template <typename R>
__global__ void k_epilogue(long long M, const double* __restrict__ eps,
                           const double* __restrict__ chi, const double* __restrict__ En,
                           const R* __restrict__ hist, double* __restrict__ Jring, int s0,
                           int jring, int n_taps, double* __restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i % M;
    const int beta = (int)(i / M);
    const long long st = 3 * M;
    const double e = En ? En[m * 3 + beta] : 0.0;
    const double ep = eps[m], ch = chi[m];
    const double j1 = Jring[jslot(s0, 1, jring, st) + i];
    const double j2 = Jring[jslot(s0, 2, jring, st) + i];
    const double j3 = Jring[jslot(s0, 3, jring, st) + i];
    double P = 0.5 / ep * j1 - ch * (double)hist[i];
    for (int l = 1; l < n_taps; ++l) P += c_taps[l] * Jring[jslot(s0, l, jring, st) + i];
    const double rhs = e - P;
    double* Jn = Jring + jslot(s0, 0, jring, st);
    if (ch > 0.0) {
        b[i] = rhs / ch;
        Jn[i] = 3.0 * j1 - 3.0 * j2 + j3;      // quadratic extrapolation as CG start
    } else {
        b[i] = 0.0;
        Jn[i] = rhs / (0.5 / ep + (n_taps > 0 ? c_taps[0] : 0.0));
    }
}

struct CGArgs {
    long long M;
    int U, V, W;
    const int* act;       // active voxels (chi > 0)
    long long nact;
    double* x;            // J_n slot (in/out)
    const double* b;
    double* r64;          // FP64 residual
    float* r;             // FP32 inner vectors
    float* p;
    float* q;
    float* e;
    const double* diag;
    double* red;          // [3][gridDim]
    double tol2;          // outer tolerance^2 (relative to ||b||^2)
    float tin2;           // inner tolerance^2 (relative to the scaled residual)
    int max_inner;        // inner iterations per refinement
    int max_iter;         // cap on total inner iterations
    int max_outer;
    int step;             // time index n (for the status record)
    int* status;          // [0] inner its, [1] flags, [2] first bad step, [3] total its, 
    double* norm2;        // ||x||^2 output
};

// the 13 offsets e > 0 (lexicographic in (ez, ey, ex)); G_0(-e) = G_0(e)
__constant__ int c_pair[13][3] = {{1, 0, 0},  {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},  {-1, -1, 1},
                                  {0, -1, 1}, {1, -1, 1}, {-1, 0, 1}, {0, 0, 1},  {1, 0, 1},
                                  {-1, 1, 1}, {0, 1, 1},  {1, 1, 1}};

// (A x)_m = diag_m x_m - sum_e G_0(e) x_{m+e} for an active voxel m, written as
// center + 13 symmetric pairs: G_0(e) (x_{m+e} + x_{m-e}).  x is zero off the active set.
template <typename T>
__device__ __forceinline__ void applyA(const CGArgs& a, const T* __restrict__ x, long long m,
                                       T o[3]) {
    const long long M = a.M;
    const int u = (int)(m % a.U), v = (int)((m / a.U) % a.V), w = (int)(m / ((long long)a.U * a.V));
    const double* S0 = c_stencil + 13 * 6;   // e = 0
    const T X0 = x[m], Y0 = x[M + m], Z0 = x[2 * M + m];
    const T d = (T)a.diag[m];
    T o0 = (d - (T)S0[0]) * X0, o1 = (d - (T)S0[1]) * Y0, o2 = (d - (T)S0[2]) * Z0;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        const int ex = c_pair[k][0], ey = c_pair[k][1], ez = c_pair[k][2];
        T sx = 0, sy = 0, sz = 0;
        {
            const int u2 = u + ex, v2 = v + ey, w2 = w + ez;
            if (u2 >= 0 && u2 < a.U && v2 >= 0 && v2 < a.V && w2 >= 0 && w2 < a.W) {
                const long long m2 = ((long long)w2 * a.V + v2) * a.U + u2;
                sx += x[m2]; sy += x[M + m2]; sz += x[2 * M + m2];
            }
        }
        {
            const int u2 = u - ex, v2 = v - ey, w2 = w - ez;
            if (u2 >= 0 && u2 < a.U && v2 >= 0 && v2 < a.V && w2 >= 0 && w2 < a.W) {
                const long long m2 = ((long long)w2 * a.V + v2) * a.U + u2;
                sx += x[m2]; sy += x[M + m2]; sz += x[2 * M + m2];
            }
        }
        const double* S = c_stencil + ((ez + 1) * 9 + (ey + 1) * 3 + (ex + 1)) * 6;
        o0 -= (T)S[0] * sx;
        o1 -= (T)S[1] * sy;
        o2 -= (T)S[2] * sz;
        if (ex != 0 && ey != 0) { o0 -= (T)S[3] * sy; o1 -= (T)S[3] * sx; }
        if (ex != 0 && ez != 0) { o0 -= (T)S[4] * sz; o2 -= (T)S[4] * sx; }
        if (ey != 0 && ez != 0) { o1 -= (T)S[5] * sz; o2 -= (T)S[5] * sy; }
    }
    o[0] = o0; o[1] = o1; o[2] = o2;
}

// block-wide sum of two values; result valid in every thread
__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sh[2][NT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < NT / 32; ++k) { s0 += sh[0][k]; s1 += sh[1][k]; }
        sh[0][0] = s0;
        sh[1][0] = s1;
    }
    __syncthreads();
    a = sh[0][0];
    b = sh[1][0];
}

// sum of the per-block partials, computed by warp 0 (fixed order: identical in every
// block) and broadcast through shared memory
__device__ __forceinline__ double grid_total(const double* red, int nb) {
    __shared__ double s_tot;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int k = threadIdx.x; k < nb; k += 32) v += __ldcg(red + k);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) s_tot = v;
    }
    __syncthreads();
    const double r = s_tot;
    __syncthreads();
    return r;
}

// Mixed-precision iterative refinement: FP64 residual r = b - A x, FP32 conjugate
// gradients for A e = r / ||r|| to a relative 1e-5 or so, x += ||r|| e; repeat until the
// FP64 residual meets tol ||b||.  All blocks take identical decisions because every
// block sums the same per-block partials in the same order.
__global__ void __launch_bounds__(NT) k_cg(CGArgs a) {
    cg::grid_group grid = cg::this_grid();
    const long long M = a.M;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gs = (long long)gridDim.x * blockDim.x;
    const int nb = gridDim.x;
    double* red0 = a.red;
    double* red1 = a.red + nb;
    double* red2 = a.red + 2 * nb;
    double bb = 0.0, rr = 0.0;
    int its = 0, outer = 0;
    bool first = true, converged = false;
    while (true) {
        // ---- FP64 residual
        double rr_p = 0.0, bb_p = 0.0;
        for (long long i = t0; i < a.nact; i += gs) {
            const long long m = a.act[i];
            double o[3];
            applyA<double>(a, a.x, m, o);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double bv = a.b[c * M + m];
                const double rv = bv - o[c];
                a.r64[c * M + m] = rv;
                rr_p += rv * rv;
                if (first) bb_p += bv * bv;
            }
        }
        block_sum2(rr_p, bb_p);
        if (threadIdx.x == 0) { red0[blockIdx.x] = rr_p; red1[blockIdx.x] = bb_p; }
        grid.sync();
        rr = grid_total(red0, nb);
        if (first) bb = grid_total(red1, nb);
        first = false;
        grid.sync();   // all blocks have read red0/red1
        if (bb == 0.0) {
            for (long long i = t0; i < a.nact; i += gs) {
                const long long m = a.act[i];
                for (int c = 0; c < 3; ++c) a.x[c * M + m] = 0.0;
            }
            rr = 0.0;
            converged = true;
            break;
        }
        if (rr <= a.tol2 * bb) { converged = true; break; }
        if (!(rr == rr) || outer >= a.max_outer || its >= a.max_iter) break;
        // ---- FP32 inner CG on the scaled residual
        const double sc = 1.0 / sqrt(rr);
        for (long long i = t0; i < a.nact; i += gs) {
            const long long m = a.act[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long k = c * M + m;
                const float rv = (float)(a.r64[k] * sc);
                a.r[k] = rv;
                a.p[k] = rv;
                a.e[k] = 0.f;
            }
        }
        double rho = 1.0;          // ||r32||^2 (scaled residual has unit norm)
        const double stop = (double)a.tin2;
        grid.sync();
        int k_in = 0;
        while (rho > stop && k_in < a.max_inner) {
            double pq = 0.0, dummy = 0.0;
            for (long long i = t0; i < a.nact; i += gs) {
                const long long m = a.act[i];
                float o[3];
                applyA<float>(a, a.p, m, o);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    a.q[c * M + m] = o[c];
                    pq += (double)a.p[c * M + m] * (double)o[c];
                }
            }
            block_sum2(pq, dummy);
            if (threadIdx.x == 0) red2[blockIdx.x] = pq;
            grid.sync();
            const float alpha = (float)(rho / grid_total(red2, nb));
            double rn = 0.0;
            for (long long i = t0; i < a.nact; i += gs) {
                const long long m = a.act[i];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long k = c * M + m;
                    a.e[k] += alpha * a.p[k];
                    const float rv = a.r[k] - alpha * a.q[k];
                    a.r[k] = rv;
                    rn += (double)rv * (double)rv;
                }
            }
            block_sum2(rn, dummy);
            if (threadIdx.x == 0) red0[blockIdx.x] = rn;
            grid.sync();
            const double rho_new = grid_total(red0, nb);
            const float beta = (float)(rho_new / rho);
            rho = rho_new;
            for (long long i = t0; i < a.nact; i += gs) {
                const long long m = a.act[i];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long k = c * M + m;
                    a.p[k] = a.r[k] + beta * a.p[k];
                }
            }
            grid.sync();
            ++k_in;
        }
        its += k_in;
        // ---- FP64 correction
        const double back = sqrt(rr);
        for (long long i = t0; i < a.nact; i += gs) {
            const long long m = a.act[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) a.x[c * M + m] += back * (double)a.e[c * M + m];
        }
        grid.sync();
        ++outer;
    }
    // norm of the solution (all voxels, active and not)
    double xx = 0.0, dummy = 0.0;
    for (long long m = t0; m < M; m += gs)
        for (int c = 0; c < 3; ++c) xx += a.x[c * M + m] * a.x[c * M + m];
    block_sum2(xx, dummy);
    grid.sync();
    if (threadIdx.x == 0) red0[blockIdx.x] = xx;
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double nx = grid_total(red0, nb);
        *a.norm2 = nx;
        a.status[0] = its;
        int flag = 0;
        if (!converged) flag |= 1;                      // not converged (or NaN)
        if (!(nx == nx) || nx > 1e300) flag |= 2;       // NaN / Inf
        if (flag && a.status[2] == 0) a.status[2] = a.step;
        a.status[1] |= flag;
        a.status[3] += its;
    }
}

// SoA slot -> AoS output [m][b]
__global__ void k_to_aos(const double* __restrict__ x, long long M, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i / 3;
    const int c = (int)(i % 3);
    out[i] = x[c * M + m];
}

// AoS [m][b] -> SoA slot
__global__ void k_from_aos(const double* __restrict__ in, long long M, double* __restrict__ x) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i / 3;
    const int c = (int)(i % 3);
    x[c * M + m] = in[i];
}

// P_{n-1} = T(1)/eps J_{n-1} + sum_{l=1}^{L-1} delta_l J_{n-l} - chi (G * J)_hist, AoS out
template <typename R>
__global__ void k_history_out(long long M, const double* __restrict__ eps,
                              const double* __restrict__ chi, const R* __restrict__ hist,
                              const double* __restrict__ Jring, int s0, int jring, int n_taps,
                              double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i % M;
    const int beta = (int)(i / M);
    const long long st = 3 * M;
    double P = 0.5 / eps[m] * Jring[jslot(s0, 1, jring, st) + i] - chi[m] * (double)hist[i];
    for (int l = 1; l < n_taps; ++l) P += c_taps[l] * Jring[jslot(s0, l, jring, st) + i];
    out[m * 3 + beta] = P;
}

}  // namespace

namespace mot {

void stencil_setup(mot_ctx* c) {
    // lag-0 elements of the 8 octant offsets in {0,1}^3 (window index 0 is lag 0 there)
    std::vector<double> oct(8 * 6);
    std::vector<double> row(6 * WIN);
    const long long U = c->U, V = c->V;
    for (int ez = 0; ez <= 1; ++ez)
        for (int ey = 0; ey <= 1; ++ey)
            for (int ex = 0; ex <= 1; ++ex) {
                for (int cc = 0; cc < 6; ++cc) oct[((ez * 2 + ey) * 2 + ex) * 6 + cc] = 0.0;
                if (ex >= c->U || ey >= c->V || ez >= c->W) continue;
                const long long o = ((long long)ez * V + ey) * U + ex;
                MOT_CUDA_TRY(cudaMemcpy(row.data(), c->tab + o * 6 * WIN, sizeof(double) * 6 * WIN,
                                        cudaMemcpyDeviceToHost));
                for (int cc = 0; cc < 6; ++cc) oct[((ez * 2 + ey) * 2 + ex) * 6 + cc] = row[cc * WIN];
            }
    for (int ez = -1; ez <= 1; ++ez)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
                const int k = ((ez + 1) * 9 + (ey + 1) * 3 + (ex + 1)) * 6;
                const double* src = &oct[((std::abs(ez) * 2 + std::abs(ey)) * 2 + std::abs(ex)) * 6];
                const int sx = ex < 0 ? -1 : 1, sy = ey < 0 ? -1 : 1, sz = ez < 0 ? -1 : 1;
                c->stencil[k + 0] = src[0];
                c->stencil[k + 1] = src[1];
                c->stencil[k + 2] = src[2];
                c->stencil[k + 3] = src[3] * sx * sy;
                c->stencil[k + 4] = src[4] * sx * sz;
                c->stencil[k + 5] = src[5] * sy * sz;
            }
    MOT_CUDA_TRY(cudaMemcpyToSymbol(c_stencil, c->stencil, sizeof(double) * 27 * 6));
    double taps[MAXTAPS] = {0};
    if (c->n_taps > MAXTAPS) throw MotError{MOT_ERR_ARG, "at most 64 FIR taps are supported"};
    for (int i = 0; i < c->n_taps; ++i) taps[i] = c->taps[i];
    MOT_CUDA_TRY(cudaMemcpyToSymbol(c_taps, taps, sizeof(double) * MAXTAPS));
    int per_sm = 0;
    MOT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg, NT, 0));
    if (per_sm < 1) throw MotError{MOT_ERR_CUDA, "CG kernel cannot be made resident"};
    const long long need = (c->M + NT - 1) / NT;
    c->cg_blocks = (int)std::min<long long>((long long)per_sm * c->nsm, std::max<long long>(need, 1));
}

template <typename R>
void epilogue(mot_ctx* c, int n, const double* En, cudaStream_t s) {
    const long long tot = 3 * c->M;
    k_epilogue<R><<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(
        c->M, c->eps, c->chi, En, hbuf<R>(c).hist_spatial, c->J, (int)slot_index(n, c->jring),
        c->jring, c->n_taps, c->rhs);
    MOT_LAUNCH_CHECK();
}

// rhs + CG for step n; ||J_n||^2 into norm2_out (device), J_n in ring slot n
void solve_step(mot_ctx* c, int n, const double* En, double* norm2_out, cudaStream_t s) {
    if (c->precision == MOT_FP64) epilogue<double>(c, n, En, s);
    else epilogue<float>(c, n, En, s);
    CGArgs a;
    a.M = c->M; a.U = c->U; a.V = c->V; a.W = c->W;
    a.act = c->active;
    a.nact = c->nact;
    a.x = c->J + slot_index(n, c->jring) * 3 * c->M;
    a.b = c->rhs;
    a.r64 = c->cg_r;
    a.r = c->cg32;
    a.p = c->cg32 + 3 * c->M;
    a.q = c->cg32 + 6 * c->M;
    a.e = c->cg32 + 9 * c->M;
    a.diag = c->cg_diag;
    a.red = c->red;
    a.tol2 = c->tol * c->tol;
    a.tin2 = 1e-10f;
    a.max_inner = 40;
    a.max_iter = c->max_iter;
    a.max_outer = 12;
    a.step = n;
    a.status = c->dstatus;
    a.norm2 = norm2_out;
    void* args[] = {&a};
    MOT_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_cg, c->cg_blocks, NT, args, 0, s));
}

void read_aos(mot_ctx* c, const double* in_dev, double* slot, cudaStream_t s) {
    const long long tot = 3 * c->M;
    k_from_aos<<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(in_dev, c->M, slot);
    MOT_LAUNCH_CHECK();
}

void history_out(mot_ctx* c, int n, double* out_dev, cudaStream_t s) {
    const long long tot = 3 * c->M;
    if (c->precision == MOT_FP64)
        k_history_out<double><<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(
            c->M, c->eps, c->chi, c->h64.hist_spatial, c->J, (int)slot_index(n, c->jring), c->jring,
            c->n_taps, out_dev);
    else
        k_history_out<float><<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(
            c->M, c->eps, c->chi, c->h32.hist_spatial, c->J, (int)slot_index(n, c->jring), c->jring,
            c->n_taps, out_dev);
    MOT_LAUNCH_CHECK();
}

void write_aos(mot_ctx* c, int n, double* out_dev, cudaStream_t s) {
    const long long tot = 3 * c->M;
    k_to_aos<<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(c->J + slot_index(n, c->jring) * 3 * c->M,
                                                       c->M, out_dev);
    MOT_LAUNCH_CHECK();
}

}  // namespace mot

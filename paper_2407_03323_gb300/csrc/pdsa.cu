// Positive definite stability analysis on the device (Sec. 5.1, Eq. Dn).
//
// The PDSA matrices D_n = sum_{i=0}^{n} (-1)^i C(ell - i, n - i) Z_i, n = 0..ell, all
// positive definite guarantee that no companion-matrix eigenvalue on the negative real
// axis lies outside the unit circle; D_ell = sum_i (-1)^i Z_i is Z(z) at z = -1.  With
// Z_i = diag(T(i)/eps + delta_i) - diag(chi) G_i (Eq. Z with the FIR taps of Sec. 6.1),
//     A_n = diag(1/chi) D_n / C(ell, n) = diag(a) - sum_i c_i G_i,
//     c_i = (-1)^i C(ell - i, n - i) / C(ell, n),
//     a_m = sum_i c_i (T(i)/(eps_m - 1) + delta_i / chi_m),
// is symmetric on the active voxels (chi > 0; the others only carry their own diagonal
// and a current that stays zero) and has the signs of D_n's eigenvalues.  Its
// Toeplitz part is one spatial convolution with the kernel sum_i c_i G_i, applied as
// in Sec. 3: forward FFT of x on the padded grid, a real symmetric 3x3 product per
// bin with the kernel spectrum, inverse FFT.
//
// Two estimates of the spectrum of A_n:
//  * a rigorous bracket from the circulant embedding (App. A): A_n = diag(a) -
//    E^T C E with C the circulant of the padded kernel and E the selection of the
//    active voxels, so by Weyl's inequality and Cauchy interlacing
//    min a - max eig C <= lambda(A_n) <= max a - min eig C, and eig C are the
//    eigenvalues of the 3x3 kernel spectrum blocks (per-bin Jacobi rotations);
//  * k steps of Lanczos from a seeded random start, either the plain three-term
//    recurrence (four vectors of memory, alpha_j and beta_j kept on the device so the
//    steps queue without host synchronisation; lost orthogonality only adds copies of
//    converged Ritz values, so k may exceed the dimension) or with full
//    reorthogonalisation (classical Gram-Schmidt applied twice against the stored
//    basis).  The Ritz values are eigenvalues of the k x k tridiagonal, found by
//    bisection on Sturm counts; each extreme Ritz value is within beta_k |y_k| of an
//    eigenvalue (y its tridiagonal eigenvector, from inverse iteration).  The smallest
//    Ritz value is an upper bound of lambda_min(A_n) (up to rounding of order
//    k eps ||A_n|| without reorthogonalisation): a clearly negative one certifies that
//    D_n is not positive definite.
#include "mot_internal.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

namespace {

constexpr int NT = 256;
constexpr int DOTV = 8;          // vectors per block row of the reorthogonalisation dots

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// a_m on active voxels, 0 elsewhere (the rows of A_n that exist)
__global__ void k_pdsa_diag(const double* __restrict__ eps, long long M, double aT, double beta,
                            double* __restrict__ a) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double e = eps[m];
    a[m] = e > 1.0 ? (aT + beta * e) / (e - 1.0) : 0.0;
}

// yhat(k) = scale * Khat(k) xhat(k) over all rfft bins, Khat from its octant
// ([noct][6]: xx yy zz xy xz yz); mirrored v / w bins flip the components odd there
__global__ void k_pdsa_mul(const double* __restrict__ spec, double2* __restrict__ xh, int Hu,
                           int Hv, int Pv, int Pw, long long nbins, double scale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbins) return;
    const int ku = (int)(i % Hu);
    const int kv = (int)((i / Hu) % Pv);
    const int kw = (int)(i / ((long long)Hu * Pv));
    const bool fv = kv >= Hv, fw = 2 * kw > Pw;
    const int ov = fv ? Pv - kv : kv;
    const int ow = fw ? Pw - kw : kw;
    const double* g = spec + (((long long)ow * Hv + ov) * Hu + ku) * 6;
    const double gxx = g[0], gyy = g[1], gzz = g[2];
    const double gxy = fv ? -g[3] : g[3];
    const double gxz = fw ? -g[4] : g[4];
    const double gyz = (fv != fw) ? -g[5] : g[5];
    const double2 x = xh[i], y = xh[nbins + i], z = xh[2 * nbins + i];
    double2 ox, oy, oz;
    ox.x = scale * (gxx * x.x + gxy * y.x + gxz * z.x);
    ox.y = scale * (gxx * x.y + gxy * y.y + gxz * z.y);
    oy.x = scale * (gxy * x.x + gyy * y.x + gyz * z.x);
    oy.y = scale * (gxy * x.y + gyy * y.y + gyz * z.y);
    oz.x = scale * (gxz * x.x + gyz * y.x + gzz * z.x);
    oz.y = scale * (gxz * x.y + gyz * y.y + gzz * z.y);
    xh[i] = ox;
    xh[nbins + i] = oy;
    xh[2 * nbins + i] = oz;
}

// y = a x - conv on active voxels, 0 elsewhere ([3][M])
__global__ void k_pdsa_combine(const double* __restrict__ a, const double* __restrict__ eps,
                               const double* __restrict__ x, const double* __restrict__ conv,
                               long long M, double* __restrict__ y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i % M;
    y[i] = eps[m] > 1.0 ? a[m] * x[i] - conv[i] : 0.0;
}

// AoS -> SoA, zero on voxels with chi = 0 (A_n acts on the active rows only)
__global__ void k_aos_to_soa(const double* __restrict__ in, const double* __restrict__ eps,
                             long long M, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i / 3;
    const int b = (int)(i % 3);
    out[b * M + m] = eps[m] > 1.0 ? in[i] : 0.0;
}

__global__ void k_soa_to_aos(const double* __restrict__ in, long long M, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i / 3;
    const int b = (int)(i % 3);
    out[i] = in[b * M + m];
}

// eigenvalues of the real symmetric 3x3 matrix by cyclic Jacobi rotations
__device__ void sym3_eigs(double A[3][3], double ev[3]) {
    for (int sweep = 0; sweep < 12; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        const double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off <= 1e-34 * dia || off == 0.0) break;
        for (int pq = 0; pq < 3; ++pq) {
            const int p = pq == 2 ? 1 : 0;
            const int q = pq == 0 ? 1 : 2;
            const double apq = A[p][q];
            if (apq == 0.0) continue;
            const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
            const int r = 3 - p - q;
            const double arp = A[r][p], arq = A[r][q];
            A[r][p] = A[p][r] = cs * arp - sn * arq;
            A[r][q] = A[q][r] = sn * arp + cs * arq;
            A[p][p] -= t * apq;
            A[q][q] += t * apq;
            A[p][q] = A[q][p] = 0.0;
        }
    }
    ev[0] = A[0][0]; ev[1] = A[1][1]; ev[2] = A[2][2];
}

// per block: min and max eigenvalue of the kernel spectrum blocks over octant bins
__global__ void k_sym3_range(const double* __restrict__ spec, long long noct,
                             double* __restrict__ part) {
    __shared__ double smin[NT / 32], smax[NT / 32];
    double lo = INFINITY, hi = -INFINITY;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < noct;
         o += (long long)gridDim.x * blockDim.x) {
        const double* g = spec + o * 6;
        double A[3][3] = {{g[0], g[3], g[4]}, {g[3], g[1], g[5]}, {g[4], g[5], g[2]}};
        double ev[3];
        sym3_eigs(A, ev);
        lo = fmin(lo, fmin(ev[0], fmin(ev[1], ev[2])));
        hi = fmax(hi, fmax(ev[0], fmax(ev[1], ev[2])));
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if ((threadIdx.x & 31) == 0) { smin[threadIdx.x >> 5] = lo; smax[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x < 32) {
        lo = threadIdx.x < NT / 32 ? smin[threadIdx.x] : INFINITY;
        hi = threadIdx.x < NT / 32 ? smax[threadIdx.x] : -INFINITY;
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (threadIdx.x == 0) { part[2 * blockIdx.x] = lo; part[2 * blockIdx.x + 1] = hi; }
    }
}

// per block: min and max of a_m and max of chi_m over active voxels
__global__ void k_diag_range(const double* __restrict__ a, const double* __restrict__ eps,
                             long long M, double* __restrict__ part) {
    __shared__ double s0[NT / 32], s1[NT / 32], s2[NT / 32];
    double lo = INFINITY, hi = -INFINITY, cmax = 0.0;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M;
         m += (long long)gridDim.x * blockDim.x) {
        const double e = eps[m];
        if (e > 1.0) {
            lo = fmin(lo, a[m]);
            hi = fmax(hi, a[m]);
            cmax = fmax(cmax, (e - 1.0) / e);
        }
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    cmax = warp_max(cmax);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s0[w] = lo; s1[w] = hi; s2[w] = cmax; }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool ok = threadIdx.x < NT / 32;
        lo = warp_min(ok ? s0[threadIdx.x] : INFINITY);
        hi = warp_max(ok ? s1[threadIdx.x] : -INFINITY);
        cmax = warp_max(ok ? s2[threadIdx.x] : 0.0);
        if (threadIdx.x == 0) {
            part[3 * blockIdx.x] = lo;
            part[3 * blockIdx.x + 1] = hi;
            part[3 * blockIdx.x + 2] = cmax;
        }
    }
}

// seeded uniform(-1, 1) start vector on the active rows (splitmix64 of seed + index)
__global__ void k_rand_vec(unsigned long long seed, const double* __restrict__ eps, long long M,
                           double* __restrict__ v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    v[i] = eps[i % M] > 1.0 ? 2.0 * u - 1.0 : 0.0;
}

// part[j][block] = partial dot(V_j, w) for j in this block row's DOTV vectors
__global__ void k_dots(const double* __restrict__ V, int nvec, long long L,
                       const double* __restrict__ w, double* __restrict__ part) {
    __shared__ double sm[DOTV][NT / 32];
    const int j0 = blockIdx.y * DOTV;
    double acc[DOTV];
#pragma unroll
    for (int j = 0; j < DOTV; ++j) acc[j] = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < L;
         r += (long long)gridDim.x * blockDim.x) {
        const double wr = w[r];
#pragma unroll
        for (int j = 0; j < DOTV; ++j)
            if (j0 + j < nvec) acc[j] = fma(V[(long long)(j0 + j) * L + r], wr, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < DOTV; ++j) {
        const double s = warp_sum(acc[j]);
        if ((threadIdx.x & 31) == 0) sm[j][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x < DOTV && j0 + (int)threadIdx.x < nvec) {
        double s = 0.0;
        for (int k = 0; k < NT / 32; ++k) s += sm[threadIdx.x][k];
        part[(long long)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
}

// h[j] = sum of the nb partials of vector j (one block per vector)
__global__ void k_sum_parts(const double* __restrict__ part, int nb, double* __restrict__ h) {
    __shared__ double sm[NT / 32];
    double s = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) s += part[(long long)blockIdx.x * nb + k];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < NT / 32 ? sm[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) h[blockIdx.x] = s;
    }
}

// w -= sum_j h[j] V_j
__global__ void k_sub_combo(double* __restrict__ w, const double* __restrict__ V,
                            const double* __restrict__ h, int nvec, long long L) {
    extern __shared__ double sh[];
    for (int j = threadIdx.x; j < nvec; j += blockDim.x) sh[j] = h[j];
    __syncthreads();
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < L;
         r += (long long)gridDim.x * blockDim.x) {
        double s = w[r];
        for (int j = 0; j < nvec; ++j) s = fma(-sh[j], V[(long long)j * L + r], s);
        w[r] = s;
    }
}

// out = w / sqrt(nrm2[0])
__global__ void k_normalise(const double* __restrict__ w, const double* __restrict__ nrm2,
                            long long L, double* __restrict__ out) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= L) return;
    out[r] = w[r] / sqrt(nrm2[0]);
}

// plain three-term Lanczos, scalars kept on the device:
// w -= beta_prev v_prev (beta_prev = sqrt(*b2prev), or 0 without a previous vector),
// part[block] = partial dot(w, v)
__global__ void k_lz_a(double* __restrict__ w, const double* __restrict__ vprev,
                       const double* __restrict__ b2prev, const double* __restrict__ v,
                       long long L, double* __restrict__ part) {
    __shared__ double sm[NT / 32];
    const double bp = b2prev ? sqrt(fmax(*b2prev, 0.0)) : 0.0;
    double acc = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < L;
         r += (long long)gridDim.x * blockDim.x) {
        double x = w[r];
        if (b2prev) x = fma(-bp, vprev[r], x);
        w[r] = x;
        acc = fma(x, v[r], acc);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = warp_sum(threadIdx.x < NT / 32 ? sm[threadIdx.x] : 0.0);
        if (threadIdx.x == 0) part[blockIdx.x] = acc;
    }
}

// w -= alpha v; part[block] = partial ||w||^2
__global__ void k_lz_b(double* __restrict__ w, const double* __restrict__ alpha,
                       const double* __restrict__ v, long long L, double* __restrict__ part) {
    __shared__ double sm[NT / 32];
    const double a = *alpha;
    double acc = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < L;
         r += (long long)gridDim.x * blockDim.x) {
        const double x = fma(-a, v[r], w[r]);
        w[r] = x;
        acc = fma(x, x, acc);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = warp_sum(threadIdx.x < NT / 32 ? sm[threadIdx.x] : 0.0);
        if (threadIdx.x == 0) part[blockIdx.x] = acc;
    }
}

// out = w / sqrt(*b2), or 0 when the norm vanished (the host stops there)
__global__ void k_lz_c(const double* __restrict__ w, const double* __restrict__ b2, long long L,
                       double* __restrict__ out) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= L) return;
    const double n2 = *b2;
    out[r] = n2 > 0.0 ? w[r] / sqrt(n2) : 0.0;
}

// ------------------------------------------------------------------ host helpers

// (n, flags) -> spectrum and diagonal of A_n in the context (cached)
void ensure_operator(mot_ctx* c, int n, int flags) {
    if (c->pdsa_n == n && c->pdsa_flags == flags) return;
    cudaStream_t s = c->stream;
    const long long M = c->M;
    if (!c->pdsa_spec) {
        MOT_CUDA_TRY(cudaMalloc(&c->pdsa_spec, sizeof(double) * 6 * c->noct));
        MOT_CUDA_TRY(cudaMalloc(&c->pdsa_a, sizeof(double) * M));
        MOT_CUDA_TRY(cudaMalloc(&c->pdsa_xhat, sizeof(double2) * 3 * c->nbins));
        MOT_CUDA_TRY(cudaMalloc(&c->pdsa_conv, sizeof(double) * 3 * M));
    }
    c->pdsa_n = c->pdsa_flags = -1;
    // c_i = (-1)^i C(ell - i, n - i) / C(ell, n), by the ratio
    // C(ell - i - 1, n - i - 1) / C(ell - i, n - i) = (n - i) / (ell - i)
    std::vector<double> w(n + 1);
    double r = 1.0;
    for (int i = 0; i <= n; ++i) {
        w[i] = (i % 2 ? -1.0 : 1.0) * r;
        if (i < n) r *= (double)(n - i) / (double)(c->ell - i);
    }
    mot::spectrum_of_combination(c, w.data(), n, (flags & MOT_PDSA_FP32_SPECTRUM) != 0,
                                 c->pdsa_spec);
    // a_m = (aT + beta eps_m) / (eps_m - 1): T(0) = T(1) = 1/2 and delta_i / chi_m =
    // delta_i eps_m / (eps_m - 1)
    const double aT = 0.5 * (w[0] + (n >= 1 ? w[1] : 0.0));
    double beta = 0.0;
    for (int i = 0; i <= n && i < c->n_taps; ++i) beta += w[i] * c->taps[i];
    k_pdsa_diag<<<nblk(M, NT), NT, 0, s>>>(c->eps, M, aT, beta, c->pdsa_a);
    MOT_LAUNCH_CHECK();
    MOT_CUDA_TRY(cudaStreamSynchronize(s));
    c->pdsa_n = n;
    c->pdsa_flags = flags;
}

// y = A_n x, both [3][M] on the device
void apply(mot_ctx* c, const double* x, double* y, cudaStream_t s) {
    const double scale = 1.0 / ((double)c->ax[0].P * c->ax[1].P * c->ax[2].P);
    mot::fft_forward<double>(c, x, c->pdsa_xhat, s, nullptr);
    k_pdsa_mul<<<nblk(c->nbins, NT), NT, 0, s>>>(c->pdsa_spec, c->pdsa_xhat, c->Hu, c->Hv,
                                                 c->ax[1].P, c->ax[2].P, c->nbins, scale);
    MOT_LAUNCH_CHECK();
    mot::fft_inverse<double>(c, c->pdsa_xhat, c->pdsa_conv, s);
    k_pdsa_combine<<<nblk(3 * c->M, NT), NT, 0, s>>>(c->pdsa_a, c->eps, x, c->pdsa_conv, c->M, y);
    MOT_LAUNCH_CHECK();
}

int grid_rows(mot_ctx* c, long long L) {
    return (int)std::max(1LL, std::min((long long)2 * std::max(c->nsm, 1), (L + NT - 1) / NT));
}

struct Scratch {
    std::vector<void*> p;
    template <typename T> T* get(long long n) {
        void* q = nullptr;
        MOT_CUDA_TRY(cudaMalloc(&q, sizeof(T) * std::max(n, 1LL)));
        p.push_back(q);
        return (T*)q;
    }
    ~Scratch() { for (void* q : p) cudaFree(q); }
};

// h[0..nvec) = V^T w (device), with partials in part ([nvec][nb])
void dots(mot_ctx* c, const double* V, int nvec, long long L, const double* w, double* part,
          double* h, cudaStream_t s) {
    const int nb = grid_rows(c, L);
    dim3 g(nb, (nvec + DOTV - 1) / DOTV);
    k_dots<<<g, NT, 0, s>>>(V, nvec, L, w, part);
    MOT_LAUNCH_CHECK();
    k_sum_parts<<<nvec, NT, 0, s>>>(part, nb, h);
    MOT_LAUNCH_CHECK();
}

// Sturm count: eigenvalues of the tridiagonal (d, e) below x
int sturm(const std::vector<double>& d, const std::vector<double>& e, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); ++i) {
        q = d[i] - x - (i ? e[i - 1] * e[i - 1] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// eigenvalues j in idx (0-based, ascending order) of the symmetric tridiagonal, by
// bisection on Sturm counts inside the Gershgorin interval
std::vector<double> tridiag_eigs(const std::vector<double>& d, const std::vector<double>& e,
                                 const std::vector<int>& idx) {
    const int m = (int)d.size();
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < m; ++i) {
        const double r = (i ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    const double span = std::max(hi - lo, 1e-300);
    lo -= 1e-12 * span;
    hi += 1e-12 * span;
    std::vector<double> out;
    for (int j : idx) {
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 4e-16 * std::max(fabs(a), fabs(b)) + 1e-300; ++it) {
            const double mid = 0.5 * (a + b);
            if (sturm(d, e, mid) > j) b = mid; else a = mid;
        }
        out.push_back(0.5 * (a + b));
    }
    return out;
}

// solve (T - sigma I) x = b for the tridiagonal T = (d, e) by Gaussian elimination with
// partial pivoting; rows kept as entries at columns (r-1, r, r+1, r+2)
std::vector<double> tridiag_solve(const std::vector<double>& d, const std::vector<double>& e,
                                  double sigma, std::vector<double> b, double tiny) {
    const int m = (int)d.size();
    std::vector<double> r0(m, 0.0), r1(m), r2(m, 0.0), r3(m, 0.0);
    for (int i = 0; i < m; ++i) {
        r1[i] = d[i] - sigma;
        if (i) r0[i] = e[i - 1];
        if (i + 1 < m) r2[i] = e[i];
    }
    for (int i = 0; i + 1 < m; ++i) {
        if (fabs(r0[i + 1]) > fabs(r1[i])) {   // swap rows i and i+1 (columns i..i+2)
            std::swap(r1[i], r0[i + 1]);
            std::swap(r2[i], r1[i + 1]);
            std::swap(r3[i], r2[i + 1]);
            std::swap(b[i], b[i + 1]);
        }
        if (r1[i] == 0.0) r1[i] = tiny;
        const double f = r0[i + 1] / r1[i];
        r1[i + 1] -= f * r2[i];
        r2[i + 1] -= f * r3[i];
        b[i + 1] -= f * b[i];
        r0[i + 1] = 0.0;
    }
    if (r1[m - 1] == 0.0) r1[m - 1] = tiny;
    std::vector<double> x(m);
    for (int i = m - 1; i >= 0; --i) {
        double s = b[i];
        if (i + 1 < m) s -= r2[i] * x[i + 1];
        if (i + 2 < m) s -= r3[i] * x[i + 2];
        x[i] = s / r1[i];
    }
    return x;
}

// last component of the unit eigenvector of T at theta (inverse iteration)
double last_component(const std::vector<double>& d, const std::vector<double>& e, double theta,
                      double norm) {
    const int m = (int)d.size();
    std::vector<double> y(m, 1.0 / sqrt((double)m));
    const double sigma = theta + 1e-13 * norm;
    for (int it = 0; it < 4; ++it) {
        std::vector<double> z = tridiag_solve(d, e, sigma, y, 1e-300 + 1e-18 * norm);
        double nz = 0.0;
        for (double v : z) nz += v * v;
        nz = sqrt(nz);
        if (!(nz > 0.0) || !std::isfinite(nz)) break;
        for (int i = 0; i < m; ++i) y[i] = z[i] / nz;
    }
    return y[m - 1];
}

template <typename F>
mot_status guard(mot_ctx* c, F&& f) {
    if (c->broken) return MOT_ERR_STATE;
    try {
        return f();
    } catch (const MotError& e) {
        c->err = e.msg;
        if (e.st == MOT_ERR_CUDA) c->broken = true;
        return e.st;
    } catch (const std::bad_alloc&) {
        c->err = "host allocation failed";
        return MOT_ERR_OOM;
    }
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

mot_status mot_pdsa_apply(mot_ctx* c, int n, int flags, const double* x, double* y) {
    if (!c) return MOT_ERR_ARG;
    if (c->precision != MOT_FP64) { c->err = "the PDSA operator needs an FP64 context"; return MOT_ERR_ARG; }
    if (n < 0 || n > c->ell || !x || !y || (flags & ~MOT_PDSA_FP32_SPECTRUM)) {
        c->err = "mot_pdsa_apply needs 0 <= n <= ell, x, y and known flags";
        return MOT_ERR_ARG;
    }
    return guard(c, [&] {
        cudaStream_t s = c->stream;
        ensure_operator(c, n, flags);
        Scratch sc;
        const long long L = 3 * c->M;
        double* xa = sc.get<double>(L);
        double* xs = sc.get<double>(L);
        double* ys = sc.get<double>(L);
        MOT_CUDA_TRY(cudaMemcpyAsync(xa, x, sizeof(double) * L,
                                     device_ptr(x) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyHostToDevice, s));
        k_aos_to_soa<<<nblk(L, NT), NT, 0, s>>>(xa, c->eps, c->M, xs);
        MOT_LAUNCH_CHECK();
        apply(c, xs, ys, s);
        k_soa_to_aos<<<nblk(L, NT), NT, 0, s>>>(ys, c->M, xa);
        MOT_LAUNCH_CHECK();
        MOT_CUDA_TRY(cudaMemcpyAsync(y, xa, sizeof(double) * L,
                                     device_ptr(y) ? cudaMemcpyDeviceToDevice
                                                   : cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
        return MOT_OK;
    });
}

mot_status mot_pdsa_bounds(mot_ctx* c, int n, int flags, double out[5]) {
    if (!c) return MOT_ERR_ARG;
    if (c->precision != MOT_FP64) { c->err = "the PDSA operator needs an FP64 context"; return MOT_ERR_ARG; }
    if (n < 0 || n > c->ell || !out || (flags & ~MOT_PDSA_FP32_SPECTRUM)) {
        c->err = "mot_pdsa_bounds needs 0 <= n <= ell, out and known flags";
        return MOT_ERR_ARG;
    }
    return guard(c, [&] {
        cudaStream_t s = c->stream;
        ensure_operator(c, n, flags);
        Scratch sc;
        const int nb = std::max(1, std::min(4 * std::max(c->nsm, 1), nblk(c->noct, NT)));
        const int nbm = std::max(1, std::min(4 * std::max(c->nsm, 1), nblk(c->M, NT)));
        double* p1 = sc.get<double>(2 * nb);
        double* p2 = sc.get<double>(3 * nbm);
        k_sym3_range<<<nb, NT, 0, s>>>(c->pdsa_spec, c->noct, p1);
        MOT_LAUNCH_CHECK();
        k_diag_range<<<nbm, NT, 0, s>>>(c->pdsa_a, c->eps, c->M, p2);
        MOT_LAUNCH_CHECK();
        std::vector<double> h1(2 * nb), h2(3 * nbm);
        MOT_CUDA_TRY(cudaMemcpyAsync(h1.data(), p1, sizeof(double) * 2 * nb,
                                     cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaMemcpyAsync(h2.data(), p2, sizeof(double) * 3 * nbm,
                                     cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
        double smin = INFINITY, smax = -INFINITY, amin = INFINITY, amax = -INFINITY, cmax = 0.0;
        for (int b = 0; b < nb; ++b) { smin = std::min(smin, h1[2 * b]); smax = std::max(smax, h1[2 * b + 1]); }
        for (int b = 0; b < nbm; ++b) {
            amin = std::min(amin, h2[3 * b]);
            amax = std::max(amax, h2[3 * b + 1]);
            cmax = std::max(cmax, h2[3 * b + 2]);
        }
        if (!(cmax > 0.0)) {
            c->err = "no voxel with eps_r > 1";
            return MOT_ERR_ARG;
        }
        out[0] = amin - smax;
        out[1] = amax - smin;
        out[2] = smin;
        out[3] = smax;
        out[4] = cmax;
        return MOT_OK;
    });
}

mot_status mot_pdsa_lanczos(mot_ctx* c, int n, int flags, int k, unsigned long long seed,
                            int n_out, double* ritz, int info[2], double extreme[4]) {
    if (!c) return MOT_ERR_ARG;
    if (c->precision != MOT_FP64) { c->err = "the PDSA operator needs an FP64 context"; return MOT_ERR_ARG; }
    const int known = MOT_PDSA_FP32_SPECTRUM | MOT_PDSA_FULL_REORTH;
    if (n < 0 || n > c->ell || k < 1 || n_out < 0 || (n_out && !ritz) || !info || !extreme ||
        (flags & ~known)) {
        c->err = "mot_pdsa_lanczos needs 0 <= n <= ell, k >= 1, n_out >= 0, ritz, info, extreme";
        return MOT_ERR_ARG;
    }
    return guard(c, [&] {
        cudaStream_t s = c->stream;
        ensure_operator(c, n, flags & MOT_PDSA_FP32_SPECTRUM);
        const long long M = c->M, L = 3 * M;
        const int g1 = nblk(L, NT);
        const int nb = grid_rows(c, L);
        Scratch sc;
        std::vector<double> alpha, beta;
        double tnorm = 0.0, last_beta = 0.0;
        if (flags & MOT_PDSA_FULL_REORTH) {
            double* V = sc.get<double>((long long)(k + 1) * L);
            double* w = sc.get<double>(L);
            double* h = sc.get<double>(k + 2);
            double* part = sc.get<double>((long long)(k + 2) * nb);
            const size_t shm = sizeof(double) * (k + 1);
            if (shm > 48 * 1024) {   // raise to the opt-in maximum (process-wide attribute)
                int dev = 0, optin = 0;
                MOT_CUDA_TRY(cudaGetDevice(&dev));
                MOT_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
                if ((int)shm > optin) {
                    c->err = "mot_pdsa_lanczos: k too large for full reorthogonalisation";
                    return MOT_ERR_ARG;
                }
                MOT_CUDA_TRY(cudaFuncSetAttribute(k_sub_combo,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
            }
            k_rand_vec<<<g1, NT, 0, s>>>(seed, c->eps, M, w);
            MOT_LAUNCH_CHECK();
            dots(c, w, 1, L, w, part, h, s);
            k_normalise<<<g1, NT, 0, s>>>(w, h, L, V);
            MOT_LAUNCH_CHECK();
            double hv[2];
            for (int j = 0; j < k; ++j) {
                apply(c, V + (long long)j * L, w, s);
                double a = 0.0;
                for (int pass = 0; pass < 2; ++pass) {   // w -= V_{0..j} (V_{0..j}^T w), twice
                    dots(c, V, j + 1, L, w, part, h, s);
                    MOT_CUDA_TRY(cudaMemcpyAsync(hv, h + j, sizeof(double), cudaMemcpyDeviceToHost, s));
                    k_sub_combo<<<nb, NT, shm, s>>>(w, V, h, j + 1, L);
                    MOT_LAUNCH_CHECK();
                    MOT_CUDA_TRY(cudaStreamSynchronize(s));
                    a += hv[0];
                }
                dots(c, w, 1, L, w, part, h + k + 1, s);
                MOT_CUDA_TRY(cudaMemcpyAsync(hv + 1, h + k + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
                MOT_CUDA_TRY(cudaStreamSynchronize(s));
                const double b = sqrt(std::max(hv[1], 0.0));
                alpha.push_back(a);
                tnorm = std::max(tnorm, fabs(a) + b + (beta.empty() ? 0.0 : beta.back()));
                last_beta = b;
                if (j + 1 == k || b <= 1e-13 * tnorm) break;    // k steps or an invariant subspace
                beta.push_back(b);
                k_normalise<<<g1, NT, 0, s>>>(w, h + k + 1, L, V + (long long)(j + 1) * L);
                MOT_LAUNCH_CHECK();
            }
        } else {
            // plain three-term recurrence: four vectors; alpha_j, beta_j^2 stay on the
            // device and are read in batches, so the steps are queued without host syncs
            double* vbuf[3] = {sc.get<double>(L), sc.get<double>(L), sc.get<double>(L)};
            double* w = sc.get<double>(L);
            double* part = sc.get<double>(nb);
            double* ad = sc.get<double>(k);
            double* b2d = sc.get<double>(k + 1);
            k_rand_vec<<<g1, NT, 0, s>>>(seed, c->eps, M, w);
            MOT_LAUNCH_CHECK();
            dots(c, w, 1, L, w, part, b2d + k, s);               // ||w||^2 of the start
            k_lz_c<<<g1, NT, 0, s>>>(w, b2d + k, L, vbuf[1]);   // v_0
            MOT_LAUNCH_CHECK();
            constexpr int BATCH = 256;
            std::vector<double> ha(BATCH), hb(BATCH);
            int done = 0;
            bool stop = false;
            while (done < k && !stop) {
                const int cnt = std::min(BATCH, k - done);
                for (int t = 0; t < cnt; ++t) {
                    const int j = done + t;
                    double* vprev = vbuf[(j + 0) % 3];
                    double* v = vbuf[(j + 1) % 3];
                    double* vnext = vbuf[(j + 2) % 3];
                    apply(c, v, w, s);
                    k_lz_a<<<nb, NT, 0, s>>>(w, vprev, j ? b2d + j - 1 : nullptr, v, L, part);
                    MOT_LAUNCH_CHECK();
                    k_sum_parts<<<1, NT, 0, s>>>(part, nb, ad + j);
                    MOT_LAUNCH_CHECK();
                    k_lz_b<<<nb, NT, 0, s>>>(w, ad + j, v, L, part);
                    MOT_LAUNCH_CHECK();
                    k_sum_parts<<<1, NT, 0, s>>>(part, nb, b2d + j);
                    MOT_LAUNCH_CHECK();
                    k_lz_c<<<g1, NT, 0, s>>>(w, b2d + j, L, vnext);
                    MOT_LAUNCH_CHECK();
                }
                MOT_CUDA_TRY(cudaMemcpyAsync(ha.data(), ad + done, sizeof(double) * cnt,
                                             cudaMemcpyDeviceToHost, s));
                MOT_CUDA_TRY(cudaMemcpyAsync(hb.data(), b2d + done, sizeof(double) * cnt,
                                             cudaMemcpyDeviceToHost, s));
                MOT_CUDA_TRY(cudaStreamSynchronize(s));
                for (int t = 0; t < cnt; ++t) {
                    const double a = ha[t], b = sqrt(std::max(hb[t], 0.0));
                    if (!std::isfinite(a) || !std::isfinite(b)) { stop = true; break; }
                    alpha.push_back(a);
                    tnorm = std::max(tnorm, fabs(a) + b + (beta.empty() ? 0.0 : beta.back()));
                    last_beta = b;
                    if ((int)alpha.size() == k || b <= 1e-13 * tnorm) { stop = true; break; }
                    beta.push_back(b);
                }
                done += cnt;
            }
        }
        const int m = (int)alpha.size();
        if (m == 0) {
            c->err = "mot_pdsa_lanczos: no step completed";
            return MOT_ERR_ARG;
        }
        const int nr = std::min(n_out, m);
        std::vector<int> idx;
        for (int i = 0; i < nr; ++i) idx.push_back(i);
        idx.push_back(0);
        idx.push_back(m - 1);
        const std::vector<double> th = tridiag_eigs(alpha, beta, idx);
        for (int i = 0; i < nr; ++i) ritz[i] = th[i];
        info[0] = nr;
        info[1] = m;
        const double tmin = th[nr], tmax = th[nr + 1];
        extreme[0] = tmin;
        extreme[1] = fabs(last_beta * last_component(alpha, beta, tmin, tnorm));
        extreme[2] = tmax;
        extreme[3] = fabs(last_beta * last_component(alpha, beta, tmax, tnorm));
        return MOT_OK;
    });
}

}  // extern "C"

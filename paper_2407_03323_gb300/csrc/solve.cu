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
// barriers (bounded waits: a barrier that is not reached in time ends the kernel with
// a timeout flag); it stops at ||r|| <= tol ||b|| or after max_iter iterations.
#include "mot_internal.cuh"

#include <type_traits>

#include <algorithm>
#include <cmath>

namespace {

constexpr int NT = 256;
constexpr int MAXTAPS = 64;
constexpr int MAXCHEB = 64;

__constant__ double c_stencil[27 * 6];   // G_0(e) for e in {-1,0,1}^3, order xx yy zz xy xz yz
// FIR taps delta_0 .. delta_{n-1} of a context, passed by value to the kernels that
// read them (several contexts with different taps may be live at once)
struct Taps {
    double d[MAXTAPS];
    int n;
};
inline Taps taps_of(const mot_ctx* c) {
    Taps t;
    for (int l = 0; l < MAXTAPS; ++l) t.d[l] = l < c->n_taps ? c->taps[l] : 0.0;
    t.n = c->n_taps;
    return t;
}

// ring slot of J_{n-l}: (s0 - l) mod jring, s0 = n mod jring, 0 <= l < jring
__device__ __forceinline__ long long jslot(int s0, int l, int jring, long long stride) {
    int sl = s0 - l;
    if (sl < 0) sl += jring;
    return (long long)sl * stride;
}

// per-voxel factors precomputed at setup (no FP64 divisions in the step):
//   f[0][m] = T(1)/eps_m = 0.5/eps_m, f[1][m] = 1/chi_m (0 if chi_m = 0),
//   f[2][m] = 1/(T(0)/eps_m + delta_0) (used where chi_m = 0), f[3][m] = chi_m
// One thread per voxel, its three components: the AoS excitation row and the four
// factors are read once and coalesced (a thread per component would read E with a
// stride of three and every factor three times).  All loads come before the stores
// (the new slot Jn lies in the same ring the loads read from, so loads placed after a
// store could not be moved ahead of it), and the FIR terms of lags 1..3 reuse them.
template <typename R>
__global__ void k_epilogue(long long M, const double* __restrict__ f, const double* __restrict__ En,
                           const R* __restrict__ hist, double* __restrict__ Jring, int s0,
                           int jring, Taps tp, double* __restrict__ b) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const long long st = 3 * M;
    const double f0 = f[m], ichi = f[M + m], f2 = f[2 * M + m], chi = f[3 * M + m];
    const double* r1 = Jring + jslot(s0, 1, jring, st);
    const double* r2 = Jring + jslot(s0, 2, jring, st);
    const double* r3 = Jring + jslot(s0, 3, jring, st);
    double* Jn = Jring + jslot(s0, 0, jring, st);
    double e[3], j1[3], j2[3], j3[3], P[3];
#pragma unroll
    for (int beta = 0; beta < 3; ++beta) {
        const long long i = beta * M + m;
        e[beta] = En ? En[m * 3 + beta] : 0.0;
        j1[beta] = r1[i];
        j2[beta] = r2[i];
        j3[beta] = r3[i];
        P[beta] = f0 * j1[beta] - chi * (double)hist[i];
    }
#pragma unroll
    for (int beta = 0; beta < 3; ++beta) {
        const long long i = beta * M + m;
        for (int l = 1; l < tp.n; ++l) {
            const double jl = l == 1 ? j1[beta] : l == 2 ? j2[beta] : l == 3 ? j3[beta]
                                                  : Jring[jslot(s0, l, jring, st) + i];
            P[beta] += tp.d[l] * jl;
        }
    }
#pragma unroll
    for (int beta = 0; beta < 3; ++beta) {
        const long long i = beta * M + m;
        const double rhs = e[beta] - P[beta];
        if (ichi > 0.0) {
            b[i] = rhs * ichi;
            Jn[i] = 3.0 * j1[beta] - 3.0 * j2[beta] + j3[beta];   // quadratic extrapolation as CG start
        } else {
            b[i] = 0.0;
            Jn[i] = rhs * f2;
        }
    }
}

struct CGArgs {
    long long M;
    int noff[27];         // neighbour e = (ez+1)*9 + (ey+1)*3 + (ex+1): m offset ex + U ey + U V ez
    const int* act;       // active voxels (chi > 0)
    const int* nmask;     // per active voxel: bit e set if neighbour e (0..26) is in the grid
    long long nact;
    int U, V, W;
    const int* tiles;     // origins (x | y << 10 | z << 20) of the 8^3 tiles with active voxels
    int ntiles;
    double* x;            // J_n slot (in/out), SoA [3][M]
    const double* b;      // rhs / chi, SoA
    const float* diag32;  // A's diagonal (T(0)/eps + delta_0)/chi, FP32 copy
    const double* diag;
    const double* chi;    // chi_m: a voxel is active (in act) iff chi_m > 0
    double* r64;          // FP64 residual, SoA
    float4* r;            // FP32 inner vectors, one float4 (x, y, z, 0) per voxel
    float4* p;
    float4* q;
    float4* e;
    // double-float residual state (FP32-history): x and b as float pairs hi + lo, and
    // the low parts of the diagonal (its high parts are diag32)
    float4* xh;
    float4* xl;
    float4* bh;
    float4* bl;
    const float* diag_lo;
    double* red;          // [3][gridDim]
    double tol2;          // outer tolerance^2 (relative to ||b||^2)
    float inv_theta;      // Chebyshev: 1 / theta, theta = (lmin + lmax) / 2
    int n_cheb;           // most Chebyshev iterations per refinement (<= MAXCHEB)
    double log_rate;      // log of the Chebyshev convergence rate (< 0)
    float c1[MAXCHEB];    // d_{k+1} = c1[k] d_k + c2[k] r_{k+1}
    float c2[MAXCHEB];
    int max_iter;         // cap on total inner iterations
    int max_outer;
    int step;             // time index n (for the status record)
    int* status;          // [0] inner its, [1] flags, [2] first bad step, [3] total its
    unsigned* bar;        // grid barrier: [0] arrivals, [1] generation, [2] abort
    long long bar_budget; // longest wait at one barrier, SM clock cycles
    double* norm2;        // ||x||^2 output
};

__constant__ float c_st32[27 * 6];   // FP32 copy of c_stencil
__constant__ float c_stl[27 * 6];    // c_stencil - c_st32 rounded to FP32 (double-float low parts)
// the 13 neighbours e > 13 pair with their mirrors 26 - e; G_0(-e) = G_0(e)

// Neighbour pair EP, 26 - EP of the 27-point stencil (G_0(-e) = G_0(e), so the pair's
// values are summed first).  Off-diagonal component (a, b) is zero unless both offset
// coordinates a and b are nonzero (parity), so face pairs take 3 products, edge pairs
// 5 and corner pairs 9.  FULL: every neighbour in the grid (no mask tests).
template <int EP, bool FULL, typename R, typename V>
__device__ __forceinline__ void stencil_pair(const R* __restrict__ S, V&& load, int mask,
                                             R& o0, R& o1, R& o2) {
    constexpr int EM = 26 - EP;
    constexpr int ex = EP % 3 - 1, ey = (EP / 3) % 3 - 1, ez = EP / 9 - 1;
    R sx = 0, sy = 0, sz = 0;
    if (FULL || (mask & (1 << EP))) load(std::integral_constant<int, EP>(), sx, sy, sz);
    if (FULL || (mask & (1 << EM))) load(std::integral_constant<int, EM>(), sx, sy, sz);
    const R* P = S + EP * 6;
    o0 -= P[0] * sx;
    o1 -= P[1] * sy;
    o2 -= P[2] * sz;
    if constexpr (ex != 0 && ey != 0) { o0 -= P[3] * sy; o1 -= P[3] * sx; }
    if constexpr (ex != 0 && ez != 0) { o0 -= P[4] * sz; o2 -= P[4] * sx; }
    if constexpr (ey != 0 && ez != 0) { o1 -= P[5] * sz; o2 -= P[5] * sy; }
}

template <bool FULL, typename R, typename V>
__device__ __forceinline__ void stencil_pairs(const R* __restrict__ S, V&& load, int mask, R& o0,
                                              R& o1, R& o2) {
    stencil_pair<14, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<15, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<16, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<17, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<18, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<19, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<20, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<21, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<22, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<23, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<24, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<25, FULL>(S, load, mask, o0, o1, o2);
    stencil_pair<26, FULL>(S, load, mask, o0, o1, o2);
}

constexpr int kAllNeighbours = (1 << 27) - 1;

// (A x)_m in FP64 for an active voxel: centre + 13 symmetric pairs
__device__ __forceinline__ void applyA64(const CGArgs& a, const double* __restrict__ x, int m,
                                         int mask, double o[3]) {
    const long long M = a.M;
    const double* S0 = c_stencil + 13 * 6;
    const double d = a.diag[m];
    double o0 = (d - S0[0]) * x[m], o1 = (d - S0[1]) * x[M + m], o2 = (d - S0[2]) * x[2 * M + m];
    auto load = [&](auto e, double& sx, double& sy, double& sz) {
        const int m2 = m + a.noff[decltype(e)::value];
        sx += x[m2];
        sy += x[M + m2];
        sz += x[2 * M + m2];
    };
    if (mask == kAllNeighbours) stencil_pairs<true>(c_stencil, load, mask, o0, o1, o2);
    else stencil_pairs<false>(c_stencil, load, mask, o0, o1, o2);
    o[0] = o0; o[1] = o1; o[2] = o2;
}

// ---- double-float residual (FP32-history mode)
// A value is a pair hi + lo of floats (about 48 significant bits).  Error-free
// transformations in FP32 with round-to-nearest intrinsics (never contracted into
// FMAs): Knuth's two-sum gives s + e = a + b exactly, and fma(a, b, -a*b) is the exact
// error of the product a*b.  Products keep the hi*lo cross terms and drop lo*lo; sums
// are accumulated without renormalising the low part.  GB300 issues FP64 at about 1/64
// of the FP32 rate, so a residual in these terms costs far fewer issue slots than in
// FP64, at a relative accuracy (~1e-14) four orders below the FP32-history tolerance.
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (oh, ol) -= (sh + sl) (xh + xl)
__device__ __forceinline__ void df_msub(float sh, float sl, float xh, float xl, float& oh,
                                        float& ol) {
    const float p = __fmul_rn(sh, xh);
    const float pe = __fadd_rn(__fmaf_rn(sh, xh, -p), __fmaf_rn(sh, xl, __fmul_rn(sl, xh)));
    float s, e;
    df_two_sum(oh, -p, s, e);
    oh = s;
    ol = __fadd_rn(ol, __fsub_rn(e, pe));
}
// (sh, sl) += (vh, vl)
__device__ __forceinline__ void df_add(float& sh, float& sl, float vh, float vl) {
    float s, e;
    df_two_sum(sh, vh, s, e);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(vl, e));
}
__device__ __forceinline__ void df_split(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// pair EP, 26 - EP in double-float (same zero pattern as stencil_pair)
template <int EP, bool FULL, typename V>
__device__ __forceinline__ void stencil_pair_df(V&& load, int mask, float* oh, float* ol) {
    constexpr int EM = 26 - EP;
    constexpr int ex = EP % 3 - 1, ey = (EP / 3) % 3 - 1, ez = EP / 9 - 1;
    float sh[3] = {0.f, 0.f, 0.f}, sl[3] = {0.f, 0.f, 0.f};
    if (FULL || (mask & (1 << EP))) load(std::integral_constant<int, EP>(), sh, sl);
    if (FULL || (mask & (1 << EM))) load(std::integral_constant<int, EM>(), sh, sl);
    const float* H = c_st32 + EP * 6;
    const float* L = c_stl + EP * 6;
    df_msub(H[0], L[0], sh[0], sl[0], oh[0], ol[0]);
    df_msub(H[1], L[1], sh[1], sl[1], oh[1], ol[1]);
    df_msub(H[2], L[2], sh[2], sl[2], oh[2], ol[2]);
    if constexpr (ex != 0 && ey != 0) {
        df_msub(H[3], L[3], sh[1], sl[1], oh[0], ol[0]);
        df_msub(H[3], L[3], sh[0], sl[0], oh[1], ol[1]);
    }
    if constexpr (ex != 0 && ez != 0) {
        df_msub(H[4], L[4], sh[2], sl[2], oh[0], ol[0]);
        df_msub(H[4], L[4], sh[0], sl[0], oh[2], ol[2]);
    }
    if constexpr (ey != 0 && ez != 0) {
        df_msub(H[5], L[5], sh[2], sl[2], oh[1], ol[1]);
        df_msub(H[5], L[5], sh[1], sl[1], oh[2], ol[2]);
    }
}

template <bool FULL, typename V>
__device__ __forceinline__ void stencil_pairs_df(V&& load, int mask, float* oh, float* ol) {
    stencil_pair_df<14, FULL>(load, mask, oh, ol);
    stencil_pair_df<15, FULL>(load, mask, oh, ol);
    stencil_pair_df<16, FULL>(load, mask, oh, ol);
    stencil_pair_df<17, FULL>(load, mask, oh, ol);
    stencil_pair_df<18, FULL>(load, mask, oh, ol);
    stencil_pair_df<19, FULL>(load, mask, oh, ol);
    stencil_pair_df<20, FULL>(load, mask, oh, ol);
    stencil_pair_df<21, FULL>(load, mask, oh, ol);
    stencil_pair_df<22, FULL>(load, mask, oh, ol);
    stencil_pair_df<23, FULL>(load, mask, oh, ol);
    stencil_pair_df<24, FULL>(load, mask, oh, ol);
    stencil_pair_df<25, FULL>(load, mask, oh, ol);
    stencil_pair_df<26, FULL>(load, mask, oh, ol);
}

// r = b - A x at an active voxel in double-float, rounded to FP32.  ch, cl: the voxel's
// x pair; dh, dl: its diagonal; bh, bl: its b pair; load(e, sh, sl) adds the x pair of
// neighbour e (compile-time index) to (sh, sl).
template <bool FULL, typename V>
__device__ __forceinline__ float4 residual_df_at(float4 ch, float4 cl, float dh, float dl,
                                                 float4 bh, float4 bl, V&& load, int mask) {
    float oh[3] = {0.f, 0.f, 0.f}, ol[3] = {0.f, 0.f, 0.f};   // o = A x
    const float* H0 = c_st32 + 13 * 6;
    const float* L0 = c_stl + 13 * 6;
    // centre block: (d - G_0(0)) x; G_0(0) is diagonal (parity)
    df_msub(-dh, -dl, ch.x, cl.x, oh[0], ol[0]);
    df_msub(-dh, -dl, ch.y, cl.y, oh[1], ol[1]);
    df_msub(-dh, -dl, ch.z, cl.z, oh[2], ol[2]);
    df_msub(H0[0], L0[0], ch.x, cl.x, oh[0], ol[0]);
    df_msub(H0[1], L0[1], ch.y, cl.y, oh[1], ol[1]);
    df_msub(H0[2], L0[2], ch.z, cl.z, oh[2], ol[2]);
    // o = (d - G_0(0)) x - sum_pairs G_0(e) (x_e + x_-e) = A x
    stencil_pairs_df<FULL>(load, mask, oh, ol);
    float r[3];
    const float bhv[3] = {bh.x, bh.y, bh.z}, blv[3] = {bl.x, bl.y, bl.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float s, e;
        df_two_sum(bhv[c], -oh[c], s, e);
        r[c] = __fadd_rn(s, __fadd_rn(__fsub_rn(blv[c], ol[c]), e));
    }
    return make_float4(r[0], r[1], r[2], 0.f);
}

// One Chebyshev pass on 8^3 tiles: d_k (with a one-voxel halo, zero outside the grid)
// is staged in shared memory, then every active voxel of the tile updates
//   e += d_k, r -= A d_k, d_{k+1} = c1 d_k + c2 r.
// Inactive voxels (diag = 0) hold zeros in every vector and are skipped.
constexpr int TT = 8;
constexpr int TH = TT + 2;
// asynchronous 16-byte global -> shared copy; zero-fills the destination when !valid
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                 "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {   // all but the newest group landed
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait0() {   // every group landed
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// halo (TH^3, zero outside the grid) of d around the tile with origin `org`
__device__ __forceinline__ void load_halo(const CGArgs& a, const float4* __restrict__ dk,
                                          float4* buf, int org) {
    const long long UV = (long long)a.U * a.V;
    const int x0 = org & 1023, y0 = (org >> 10) & 1023, z0 = org >> 20;
    for (int h = threadIdx.x; h < TH * TH * TH; h += blockDim.x) {
        const int hx = h % TH, hy = (h / TH) % TH, hz = h / (TH * TH);
        const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
        const bool in = x >= 0 && x < a.U && y >= 0 && y < a.V && z >= 0 && z < a.W;
        cp_async16(&buf[h], in ? dk + ((long long)z * UV + (long long)y * a.U + x) : dk, in);
    }
}

// One Chebyshev iteration over the tiles of this block: r -= A d_k, e += d_k (e = d_0
// on the first iteration, so e needs no clearing), d_{k+1} = c1 d_k + c2 r.  The halo of the next tile is copied into the other shared
// buffer while the current one is computed, and each thread loads its voxels' own
// e, r and diagonal before waiting for the halo.
constexpr int kVoxPerThread = TT * TT * TT / NT;
static_assert(kVoxPerThread * NT == TT * TT * TT, "tile voxels per thread");
__device__ __forceinline__ void cheb_pass_tiled(const CGArgs& a, const float4* __restrict__ dk,
                                                float4* __restrict__ dn, float c1, float c2,
                                                bool first, float4 (*sd)[TH * TH * TH]) {
    const long long UV = (long long)a.U * a.V;
    int tile = blockIdx.x;
    if (tile < a.ntiles) load_halo(a, dk, sd[0], a.tiles[tile]);
    cp_async_commit();
    for (int it = 0; tile < a.ntiles; ++it, tile += gridDim.x) {
        const int next = tile + gridDim.x;
        if (next < a.ntiles) load_halo(a, dk, sd[(it + 1) & 1], a.tiles[next]);
        cp_async_commit();
        const int org = a.tiles[tile];
        const int x0 = org & 1023, y0 = (org >> 10) & 1023, z0 = org >> 20;
        long long mv[kVoxPerThread];
        float dgv[kVoxPerThread];
        float4 ev[kVoxPerThread], rv[kVoxPerThread];
#pragma unroll
        for (int v = 0; v < kVoxPerThread; ++v) {
            const int q = threadIdx.x + v * NT;
            const int lx = q % TT, ly = (q / TT) % TT, lz = q / (TT * TT);
            const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
            mv[v] = -1;
            dgv[v] = 0.f;
            if (x < a.U && y < a.V && z < a.W) {
                const long long m = (long long)z * UV + (long long)y * a.U + x;
                dgv[v] = a.diag32[m];
                if (dgv[v] != 0.f) {
                    mv[v] = m;
                    ev[v] = first ? make_float4(0.f, 0.f, 0.f, 0.f) : a.e[m];
                    rv[v] = a.r[m];
                }
            }
        }
        cp_async_wait1();
        __syncthreads();
        const float4* sb = sd[it & 1];
#pragma unroll
        for (int v = 0; v < kVoxPerThread; ++v) {
            if (mv[v] < 0) continue;
            const int q = threadIdx.x + v * NT;
            const int lx = q % TT, ly = (q / TT) % TT, lz = q / (TT * TT);
            const int hc = ((lz + 1) * TH + (ly + 1)) * TH + (lx + 1);
            const float dg = dgv[v];
            const float* S0 = c_st32 + 13 * 6;
            const float4 c = sb[hc];
            float o0 = (dg - S0[0]) * c.x, o1 = (dg - S0[1]) * c.y, o2 = (dg - S0[2]) * c.z;
            auto load = [&](auto e, float& sx, float& sy, float& sz) {
                constexpr int E = decltype(e)::value;
                constexpr int off = ((E / 9 - 1) * TH + ((E / 3) % 3 - 1)) * TH + (E % 3 - 1);
                const float4 v = sb[hc + off];
                sx += v.x;
                sy += v.y;
                sz += v.z;
            };
            stencil_pairs<true>(c_st32, load, 0, o0, o1, o2);
            float4 e = ev[v], r = rv[v];
            e.x += c.x; e.y += c.y; e.z += c.z;
            r.x -= o0; r.y -= o1; r.z -= o2;
            const long long m = mv[v];
            a.e[m] = e;
            a.r[m] = r;
            dn[m] = make_float4(c1 * c.x + c2 * r.x, c1 * c.y + c2 * r.y, c1 * c.z + c2 * r.z, 0.f);
        }
        __syncthreads();
    }
}

// Double-float residual pass on the 8^3 tiles (FP32-history): the two halves of the
// shared halo buffer hold the hi and lo parts of x around the tile (zero outside the
// grid and on inactive voxels, so no neighbour mask is needed).  Writes r (rounded to
// FP32) and the first Chebyshev direction d_0 = r / theta on active voxels and adds
// |r|^2 (and, on the first pass, |b|^2 in FP64) to the thread's partial sums.
__device__ __forceinline__ void residual_df_tiled(const CGArgs& a, float4 (*sd)[TH * TH * TH],
                                                  double& rr_p, double& bb_p, bool first) {
    const long long UV = (long long)a.U * a.V;
    const long long M = a.M;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int org = a.tiles[tile];
        load_halo(a, a.xh, sd[0], org);
        load_halo(a, a.xl, sd[1], org);
        cp_async_commit();
        const int x0 = org & 1023, y0 = (org >> 10) & 1023, z0 = org >> 20;
        long long mv[kVoxPerThread];
        float dhv[kVoxPerThread], dlv[kVoxPerThread];
        float4 bhv[kVoxPerThread], blv[kVoxPerThread];
#pragma unroll
        for (int v = 0; v < kVoxPerThread; ++v) {
            const int q = threadIdx.x + v * NT;
            const int x = x0 + q % TT, y = y0 + (q / TT) % TT, z = z0 + q / (TT * TT);
            mv[v] = -1;
            if (x < a.U && y < a.V && z < a.W) {
                const long long m = (long long)z * UV + (long long)y * a.U + x;
                dhv[v] = a.diag32[m];
                if (dhv[v] != 0.f) {
                    mv[v] = m;
                    dlv[v] = a.diag_lo[m];
                    bhv[v] = a.bh[m];
                    blv[v] = a.bl[m];
                    if (first) {
                        const double b0 = a.b[m], b1 = a.b[M + m], b2 = a.b[2 * M + m];
                        bb_p += b0 * b0 + b1 * b1 + b2 * b2;
                    }
                }
            }
        }
        cp_async_wait0();
        __syncthreads();
#pragma unroll
        for (int v = 0; v < kVoxPerThread; ++v) {
            if (mv[v] < 0) continue;
            const int q = threadIdx.x + v * NT;
            const int hc = ((q / (TT * TT) + 1) * TH + ((q / TT) % TT + 1)) * TH + (q % TT + 1);
            auto load = [&](auto e, float* sh, float* sl) {
                constexpr int E = decltype(e)::value;
                constexpr int off = ((E / 9 - 1) * TH + ((E / 3) % 3 - 1)) * TH + (E % 3 - 1);
                const float4 vh = sd[0][hc + off], vl = sd[1][hc + off];
                df_add(sh[0], sl[0], vh.x, vl.x);
                df_add(sh[1], sl[1], vh.y, vl.y);
                df_add(sh[2], sl[2], vh.z, vl.z);
            };
            const float4 r = residual_df_at<true>(sd[0][hc], sd[1][hc], dhv[v], dlv[v], bhv[v],
                                                  blv[v], load, 0);
            rr_p += (double)r.x * r.x + (double)r.y * r.y + (double)r.z * r.z;
            a.r[mv[v]] = r;
            a.p[mv[v]] = make_float4(r.x * a.inv_theta, r.y * a.inv_theta, r.z * a.inv_theta, 0.f);
        }
        __syncthreads();
    }
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
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;   // four independent loads in flight
        int k = threadIdx.x;
        for (; k + 96 < nb; k += 128) {
            v0 += __ldcg(red + k);
            v1 += __ldcg(red + k + 32);
            v2 += __ldcg(red + k + 64);
            v3 += __ldcg(red + k + 96);
        }
        for (; k < nb; k += 32) v0 += __ldcg(red + k);
        double v = (v0 + v1) + (v2 + v3);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) s_tot = v;
    }
    __syncthreads();
    const double r = s_tot;
    __syncthreads();
    return r;
}

// Grid-wide barrier of a cooperative launch (every block resident) with a bounded wait.
// After a block-level barrier, thread 0 of each block publishes the block's writes
// (fence), arrives on a counter and, unless it is the last to arrive, waits for the
// generation word to change; the last block resets the counter and advances the
// generation.  A wait longer than `budget` SM clock cycles (a block that never
// arrives) sets the abort word and the timeout flag (4) in status[1] with the step in
// status[2]; blocks that see the abort word leave at once.  Returns false when the
// caller must return: the kernel ends without touching the solution any further.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ bool grid_barrier(unsigned* bar, long long budget, int* status, int step) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = ld_acquire_gpu(bar + 2) == 0;
        if (ok) {
            const unsigned gen = ld_acquire_gpu(bar + 1);
            __threadfence();
            if (atomicAdd(bar, 1u) == gridDim.x - 1) {
                bar[0] = 0u;
                st_release_gpu(bar + 1, gen + 1u);
            } else {
                const long long t0 = clock64();
                while (ld_acquire_gpu(bar + 1) == gen) {
                    if (ld_acquire_gpu(bar + 2) != 0u) { ok = 0; break; }
                    if (clock64() - t0 > budget) {
                        atomicExch(bar + 2, 1u);
                        atomicOr(status + 1, 4);
                        atomicCAS(status + 2, 0, step);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// for i = t0, t0 + gs, ... < n: U indices per round, ld(i) for all of them before
// st(i, value) for any (the loads of a round are independent requests in flight)
template <int U, typename Ld, typename St>
__device__ __forceinline__ void grid_loop(long long t0, long long n, long long gs, Ld&& ld,
                                          St&& st) {
    for (long long i0 = t0; i0 < n; i0 += U * gs) {
        decltype(ld(0LL)) v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * gs < n) v[u] = ld(i0 + u * gs);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * gs < n) st(i0 + u * gs, v[u]);
    }
}

// Check of the barrier's bounded wait: every block passes `rounds` barriers, except the
// block `absent` (>= 0), which returns at once; the others' wait then runs out.
// w[1] flags, w[2] the round of a timeout, w[4..6] the barrier, w[7] blocks that
// passed every round.
__global__ void __launch_bounds__(NT) k_barrier_check(int* w, long long budget, int rounds,
                                                      int absent) {
    if ((int)blockIdx.x == absent) return;
    for (int r = 1; r <= rounds; ++r)
        if (!grid_barrier(reinterpret_cast<unsigned*>(w + 4), budget, w, r)) return;
    if (threadIdx.x == 0) atomicAdd(w + 7, 1);
}

// Mixed-precision iterative refinement: FP64 residual r = b - A x, FP32 conjugate
// gradients for A e = r / ||r|| to a relative ~1e-5, x += ||r|| e; repeat until the
// FP64 residual meets tol ||b||.  All blocks take identical decisions because every
// block sums the same per-block partials in the same order.  DF: the residual is
// evaluated in double-float arithmetic on float-pair copies of x and b (FP32-history
// mode); x is split at entry, corrected in pairs and merged back to FP64 at exit.
template <bool DF>
__global__ void __launch_bounds__(NT, 3) k_cg(const __grid_constant__ CGArgs a) {
    auto gsync = [&] { return grid_barrier(a.bar, a.bar_budget, a.status, a.step); };
    __shared__ float4 sd[2][TH * TH * TH];        // tile halos of the tiled passes
    const long long M = a.M;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gs = (long long)gridDim.x * blockDim.x;
    const int nb = gridDim.x;
    double* red0 = a.red;
    double* red1 = a.red + nb;
    double bb = 0.0, rr = 0.0;
    int its = 0, outer = 0;
    bool first = true, converged = false, zeroed = false, nonfinite = false;
    // grid-stride loops over the active voxels (or all voxels) take four indices per
    // thread per round and issue all their loads before the first store, so that a
    // thread has several independent memory requests in flight
    struct XB { int m; double x0, x1, x2, b0, b1, b2; };
    struct RF { int m; float4 r; };
    struct RD { int m; double r0, r1, r2; };
    struct EHL { int m; float4 e, h, l; };
    struct EX3 { int m; float4 e; double x0, x1, x2; };
    struct X3 { bool pair; double x0, x1, x2; };
    if (DF) {
        grid_loop<1>(t0, a.nact, gs,
            [&](long long i) {
                XB v;
                v.m = a.act[i];
                v.x0 = a.x[v.m]; v.x1 = a.x[M + v.m]; v.x2 = a.x[2 * M + v.m];
                v.b0 = a.b[v.m]; v.b1 = a.b[M + v.m]; v.b2 = a.b[2 * M + v.m];
                return v;
            },
            [&](long long, const XB& v) {
                float4 h, l;
                df_split(v.x0, h.x, l.x);
                df_split(v.x1, h.y, l.y);
                df_split(v.x2, h.z, l.z);
                h.w = l.w = 0.f;
                a.xh[v.m] = h;
                a.xl[v.m] = l;
                df_split(v.b0, h.x, l.x);
                df_split(v.b1, h.y, l.y);
                df_split(v.b2, h.z, l.z);
                a.bh[v.m] = h;
                a.bl[v.m] = l;
            });
        if (!gsync()) return;
    }
    while (true) {
        // ---- residual (FP64, or double-float rounded to FP32 with d_0 = r / theta)
        double rr_p = 0.0, bb_p = 0.0;
        if (DF) residual_df_tiled(a, sd, rr_p, bb_p, first);
        for (long long i = t0; !DF && i < a.nact; i += gs) {
            const int m = a.act[i];
            if (first) {
                const double b0 = a.b[m], b1 = a.b[M + m], b2 = a.b[2 * M + m];
                bb_p += b0 * b0 + b1 * b1 + b2 * b2;
            }
            {
                double o[3];
                applyA64(a, a.x, m, a.nmask[i], o);
                const double r0 = a.b[m] - o[0], r1 = a.b[M + m] - o[1], r2 = a.b[2 * M + m] - o[2];
                rr_p += r0 * r0 + r1 * r1 + r2 * r2;
                a.r64[m] = r0;
                a.r64[M + m] = r1;
                a.r64[2 * M + m] = r2;
            }
        }
        block_sum2(rr_p, bb_p);
        if (threadIdx.x == 0) { red0[blockIdx.x] = rr_p; red1[blockIdx.x] = bb_p; }
        if (!gsync()) return;
        rr = grid_total(red0, nb);
        if (first) bb = grid_total(red1, nb);
        first = false;
        // red0 / red1 are written next after at least one more barrier (the next
        // residual follows the Chebyshev passes; the final norm follows the merge or
        // its own barrier), so no barrier is needed here for their readers
        if (!(rr <= 1e300) || !(bb <= 1e300)) {
            // NaN or Inf in the right-hand side (or the start): no iteration can help;
            // J_n is returned as NaN so that the monitor and the caller see it
            const double qnan = __longlong_as_double(0x7ff8000000000000LL);
            for (long long i = t0; i < a.nact; i += gs) {
                const int m = a.act[i];
                a.x[m] = qnan; a.x[M + m] = qnan; a.x[2 * M + m] = qnan;
            }
            nonfinite = true;
            break;
        }
        if (bb == 0.0) {
            for (long long i = t0; i < a.nact; i += gs) {
                const int m = a.act[i];
                a.x[m] = 0.0; a.x[M + m] = 0.0; a.x[2 * M + m] = 0.0;
            }
            rr = 0.0;
            converged = zeroed = true;
            break;
        }
        if (rr <= a.tol2 * bb) { converged = true; break; }
        if (outer >= a.max_outer || its >= a.max_iter) break;
        // ---- FP32 Chebyshev iteration for A e = r (r holds the FP32 residual).
        // One fused pass per iteration (apply to d_k, update e, r, d_{k+1}) and one grid
        // barrier; d is double-buffered because neighbours read d_k during the pass.
        // iterations for the reduction still needed (with a factor 10 of margin), never
        // asking for more than FP32 can deliver in one refinement (5e-6)
        const double need = fmax(0.1 * sqrt(a.tol2 * bb / rr), 5e-6);
        const int n_it = min(a.n_cheb, max(3, (int)ceil(log(0.5 * need) / a.log_rate)));
        // The double-float residual is already an FP32 vector with d_0 beside it; it is
        // iterated as it is unless its norm is far from 1 (FP32 range).  Otherwise (and
        // always for the FP64 residual) r is first scaled to unit norm in FP64, so that
        // a tiny residual cannot underflow in FP32, and e is scaled back by ||r||.
        const bool scaled = !DF || !(rr >= 1e-40 && rr <= 1e40);
        const double sc = scaled ? 1.0 / sqrt(rr) : 1.0;
        if (scaled) {
            const float sc32 = (float)sc;
            if constexpr (DF) {
                grid_loop<4>(t0, a.nact, gs,
                    [&](long long i) { const int m = a.act[i]; return RF{m, a.r[m]}; },
                    [&](long long, const RF& v) {
                        const float4 rv = make_float4(v.r.x * sc32, v.r.y * sc32, v.r.z * sc32, 0.f);
                        a.r[v.m] = rv;
                        a.p[v.m] = make_float4(rv.x * a.inv_theta, rv.y * a.inv_theta,
                                               rv.z * a.inv_theta, 0.f);
                    });
            } else {
                grid_loop<4>(t0, a.nact, gs,
                    [&](long long i) {
                        const int m = a.act[i];
                        return RD{m, a.r64[m], a.r64[M + m], a.r64[2 * M + m]};
                    },
                    [&](long long, const RD& v) {
                        const float4 rv = make_float4((float)(v.r0 * sc), (float)(v.r1 * sc),
                                                      (float)(v.r2 * sc), 0.f);
                        a.r[v.m] = rv;
                        a.p[v.m] = make_float4(rv.x * a.inv_theta, rv.y * a.inv_theta,
                                               rv.z * a.inv_theta, 0.f);
                    });
            }
            if (!gsync()) return;
        }
        float4* dk = a.p;
        float4* dn = a.q;
        for (int k = 0; k < n_it; ++k) {
            cheb_pass_tiled(a, dk, dn, a.c1[k], a.c2[k], k == 0, sd);
            if (!gsync()) return;
            float4* t = dk; dk = dn; dn = t;
        }
        its += n_it;
        // ---- correction x += (1 / sc) e (FP64, or in float pairs)
        const double back = 1.0 / sc;
        float bkh, bkl;
        df_split(back, bkh, bkl);
        if constexpr (DF) {
            grid_loop<1>(t0, a.nact, gs,
                [&](long long i) {
                    const int m = a.act[i];
                    return EHL{m, a.e[m], a.xh[m], a.xl[m]};
                },
                [&](long long, const EHL& v) {
                    const float ec[3] = {v.e.x, v.e.y, v.e.z};
                    float hc[3] = {v.h.x, v.h.y, v.h.z}, lc[3] = {v.l.x, v.l.y, v.l.z};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float p = __fmul_rn(bkh, ec[c]);
                        const float pe = __fmaf_rn(bkh, ec[c], -p) + __fmul_rn(bkl, ec[c]);
                        df_add(hc[c], lc[c], p, pe);
                    }
                    a.xh[v.m] = make_float4(hc[0], hc[1], hc[2], 0.f);
                    a.xl[v.m] = make_float4(lc[0], lc[1], lc[2], 0.f);
                });
        } else {
            grid_loop<4>(t0, a.nact, gs,
                [&](long long i) {
                    const int m = a.act[i];
                    return EX3{m, a.e[m], a.x[m], a.x[M + m], a.x[2 * M + m]};
                },
                [&](long long, const EX3& v) {
                    a.x[v.m] = v.x0 + back * (double)v.e.x;
                    a.x[M + v.m] = v.x1 + back * (double)v.e.y;
                    a.x[2 * M + v.m] = v.x2 + back * (double)v.e.z;
                });
        }
        if (!gsync()) return;
        ++outer;
    }
    // norm of the solution (all voxels, active and not).  In the double-float mode the
    // same pass merges x = hi + lo back to FP64 at the active voxels (their pairs were
    // last written before the final residual's barrier; a voxel's x is read and
    // written by its own thread only); elsewhere x is read as it is, and x written by
    // other blocks without a barrier since (zeroed or non-finite start) needs one
    const bool merge = DF && !zeroed && !nonfinite;
    if ((zeroed || nonfinite) && !gsync()) return;
    double xx = 0.0, dummy = 0.0;
    grid_loop<4>(t0, M, gs,
        [&](long long m) {
            X3 v;
            v.pair = merge && a.chi[m] > 0.0;
            if (v.pair) {
                const float4 h = a.xh[m], l = a.xl[m];
                v.x0 = (double)h.x + (double)l.x;
                v.x1 = (double)h.y + (double)l.y;
                v.x2 = (double)h.z + (double)l.z;
            } else {
                v.x0 = a.x[m]; v.x1 = a.x[M + m]; v.x2 = a.x[2 * M + m];
            }
            return v;
        },
        [&](long long m, const X3& v) {
            if (v.pair) { a.x[m] = v.x0; a.x[M + m] = v.x1; a.x[2 * M + m] = v.x2; }
            xx += v.x0 * v.x0 + v.x1 * v.x1 + v.x2 * v.x2;
        });
    block_sum2(xx, dummy);
    // the third partial-sum array: nothing in this launch has read it, so no barrier
    // is needed before the write (red0 may still be read for the last residual norm)
    double* red2 = a.red + 2 * nb;
    if (threadIdx.x == 0) red2[blockIdx.x] = xx;
    if (!gsync()) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double nx = grid_total(red2, nb);
        *a.norm2 = nx;
        a.status[0] = its;
        int flag = 0;
        if (!converged && !nonfinite) flag |= 1;        // not converged
        if (nonfinite || !(nx == nx) || nx > 1e300) flag |= 2;   // NaN / Inf
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

// ---------------------------------------------------------------- adjoint march
// In adjoint time tau = N + 1 - n the ring holds lambda.  With mu = chi lambda,
//   Z_0^T lambda_n = g_n - sum_{l>=1} Z_l^T lambda_{n+l},
//   Z_l^T lambda = (T(l)/eps + delta_l) lambda - G_l * (chi lambda)      (G_l^T = G_l),
// and Z_0^T lambda = A mu with the same symmetric A as the forward solve.
template <typename R>
__global__ void k_epilogue_adj(long long M, const double* __restrict__ f,
                               const double* __restrict__ g, const R* __restrict__ hist,
                               double* __restrict__ Lring, int s0, int jring, Taps tp,
                               double* __restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i % M;
    const int beta = (int)(i / M);
    const long long st = 3 * M;
    const double l1 = Lring[jslot(s0, 1, jring, st) + i];
    const double l2 = Lring[jslot(s0, 2, jring, st) + i];
    const double l3 = Lring[jslot(s0, 3, jring, st) + i];
    double P = f[m] * l1 - (double)hist[i];
    for (int l = 1; l < tp.n; ++l) P += tp.d[l] * Lring[jslot(s0, l, jring, st) + i];
    const double rhs = g[m * 3 + beta] - P;
    double* Ln = Lring + jslot(s0, 0, jring, st);
    const double chi = f[3 * M + m];
    b[i] = rhs;                                        // A mu = rhs on active voxels
    // the solve's iterate must vanish off the active set; vacuum voxels get their
    // lambda after the solve (k_adj_post), when mu is known
    Ln[i] = chi > 0.0 ? chi * (3.0 * l1 - 3.0 * l2 + l3) : 0.0;
}

// lambda = mu / chi on active voxels; on vacuum voxels (chi = 0) the row of Z_0^T reads
// (T(0) + delta_0) lambda_m - (G_0 * mu)_m = rhs_m, so lambda_m = (rhs_m + (G_0 * mu)_m)
// / (T(0) + delta_0).  Gradient accumulation on active voxels:
//   dO/dchi_m += lambda_n,m . (1/chi_m) sum_l (T(l) + delta_l) J_{n-l,m}
// (the chi-derivative of row m of the forward system, simplified with that row's own
// equation), and optional AoS output of lambda_n.  Two launches: the first turns mu
// into lambda on active voxels only after the second has read mu around vacuum ones.
__global__ void k_adj_vacuum(long long M, int U, int V, int W, const double* __restrict__ f,
                             const double* __restrict__ mu, const double* __restrict__ rhs,
                             double* __restrict__ lam_vac) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    if (f[M + m] > 0.0) return;
    const int u = (int)(m % U), v = (int)((m / U) % V), w = (int)(m / ((long long)U * V));
    double o[3] = {0.0, 0.0, 0.0};
    for (int ez = -1; ez <= 1; ++ez)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
                const int u2 = u + ex, v2 = v + ey, w2 = w + ez;
                if (u2 < 0 || u2 >= U || v2 < 0 || v2 >= V || w2 < 0 || w2 >= W) continue;
                const long long m2 = ((long long)w2 * V + v2) * U + u2;
                const double* S = c_stencil + ((ez + 1) * 9 + (ey + 1) * 3 + (ex + 1)) * 6;
                const double X = mu[m2], Y = mu[M + m2], Z = mu[2 * M + m2];
                o[0] += S[0] * X + S[3] * Y + S[4] * Z;
                o[1] += S[3] * X + S[1] * Y + S[5] * Z;
                o[2] += S[4] * X + S[5] * Y + S[2] * Z;
            }
    for (int beta = 0; beta < 3; ++beta)
        lam_vac[beta * M + m] = (rhs[beta * M + m] + o[beta]) * f[2 * M + m];
}

__global__ void k_adj_post(long long M, const double* __restrict__ f, double* __restrict__ Ln,
                           const double* __restrict__ lam_vac, const double* __restrict__ J,
                           int j_first, int n, Taps tp, double* __restrict__ grad_chi,
                           double* __restrict__ lam_out) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double ichi = f[M + m];
    double gsum = 0.0;
    for (int beta = 0; beta < 3; ++beta) {
        double lam;
        if (ichi > 0.0) {
            lam = Ln[beta * M + m] * ichi;
            double q = 0.0;
            const int L = tp.n > 2 ? tp.n : 2;
            for (int l = 0; l < L && n - l >= 1; ++l) {   // J[0] holds step j_first
                const double w = (l < 2 ? 0.5 : 0.0) + (l < tp.n ? tp.d[l] : 0.0);
                q += w * J[((long long)(n - l - j_first) * M + m) * 3 + beta];
            }
            gsum += lam * q * ichi;
        } else {
            lam = lam_vac[beta * M + m];
        }
        Ln[beta * M + m] = lam;
        if (lam_out) lam_out[m * 3 + beta] = lam;
    }
    grad_chi[m] += gsum;
}

// P_{n-1} = T(1)/eps J_{n-1} + sum_{l=1}^{L-1} delta_l J_{n-l} - chi (G * J)_hist, AoS out
template <typename R>
__global__ void k_history_out(long long M, const double* __restrict__ eps,
                              const double* __restrict__ chi, const R* __restrict__ hist,
                              const double* __restrict__ Jring, int s0, int jring, Taps tp,
                              double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    const long long m = i % M;
    const int beta = (int)(i / M);
    const long long st = 3 * M;
    double P = 0.5 / eps[m] * Jring[jslot(s0, 1, jring, st) + i] - chi[m] * (double)hist[i];
    for (int l = 1; l < tp.n; ++l) P += tp.d[l] * Jring[jslot(s0, l, jring, st) + i];
    out[m * 3 + beta] = P;
}

// y = A x (FP64) on active voxels, for the setup-time eigenvalue estimate
__global__ void k_apply64(const __grid_constant__ CGArgs a, const double* __restrict__ x,
                          double* __restrict__ y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nact) return;
    const int m = a.act[i];
    double o[3];
    applyA64(a, x, m, a.nmask[i], o);
    y[m] = o[0];
    y[a.M + m] = o[1];
    y[2 * a.M + m] = o[2];
}

// partial dot products per block
__global__ void k_dot(const double* __restrict__ x, const double* __restrict__ y, long long n,
                      double* __restrict__ part) {
    double s = 0.0, d = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        s += x[i] * y[i];
    block_sum2(s, d);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// w = w - alpha v - beta u
__global__ void k_axpy2(double* __restrict__ w, const double* __restrict__ v, double alpha,
                        const double* __restrict__ u, double beta, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] -= alpha * v[i] + beta * u[i];
}

__global__ void k_scale(double* __restrict__ w, double s, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] *= s;
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
                // component (a, b), a != b, is odd in d_a and in d_b: exactly zero when
                // either offset coordinate is 0 (the stencil kernels skip those products)
                c->stencil[k + 3] = (ex && ey) ? src[3] * sx * sy : 0.0;
                c->stencil[k + 4] = (ex && ez) ? src[4] * sx * sz : 0.0;
                c->stencil[k + 5] = (ey && ez) ? src[5] * sy * sz : 0.0;
            }
    // The stencil constants are shared by every context on the device: G_0 at offsets
    // |d_i| <= 1 depends on the unit voxel only, so all contexts compute the same
    // values.  A grid of extent 1 along some axis lacks those neighbours (its entries
    // are zero, and masked out of its own stencil), so it writes the constants only
    // while no complete stencil is there.
    const bool complete = c->U > 1 && c->V > 1 && c->W > 1;
    int dev = 0;
    MOT_CUDA_TRY(cudaGetDevice(&dev));
    static bool have_complete[64] = {};
    if (complete || dev >= 64 || !have_complete[dev]) {
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_stencil, c->stencil, sizeof(double) * 27 * 6));
        float st32[27 * 6];
        float stl[27 * 6];
        for (int k = 0; k < 27 * 6; ++k) {
            st32[k] = (float)c->stencil[k];
            stl[k] = (float)(c->stencil[k] - (double)st32[k]);
        }
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_st32, st32, sizeof st32));
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_stl, stl, sizeof stl));
        if (complete && dev < 64) have_complete[dev] = true;
    }
    int noff[27];
    for (int ez = -1; ez <= 1; ++ez)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex)
                noff[(ez + 1) * 9 + (ey + 1) * 3 + (ex + 1)] = ex + c->U * (ey + c->V * ez);
    for (int e = 0; e < 27; ++e) c->noff[e] = noff[e];
    if (c->n_taps > MAXTAPS) throw MotError{MOT_ERR_ARG, "at most 64 FIR taps are supported"};
    int per_sm = 0;
    if (c->precision == MOT_FP64)
        MOT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg<false>, NT, 0));
    else
        MOT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg<true>, NT, 0));
    if (per_sm < 1) throw MotError{MOT_ERR_CUDA, "CG kernel cannot be made resident"};
    const long long need = (c->M + NT - 1) / NT;
    c->cg_blocks = (int)std::min<long long>((long long)per_sm * c->nsm, std::max<long long>(need, 1));
    int khz = 0;
    MOT_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device));
    c->bar_budget = (long long)(kBarrierBudgetS * 1e3 * std::max(khz, 1000000));
}

namespace {

// number of eigenvalues of the symmetric tridiagonal (al, be) below x (Sturm count)
int sturm_count(const std::vector<double>& al, const std::vector<double>& be, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < al.size(); ++i) {
        const double b2 = i ? be[i] * be[i] : 0.0;
        q = al[i] - x - (i ? b2 / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

double tridiag_eig(const std::vector<double>& al, const std::vector<double>& be, int k,
                   double lo, double hi) {
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(al, be, mid) > k) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

// Spectral bounds of A = diag(1/chi) Z_0 on the active voxels by 40 Lanczos steps from a
// seeded start vector, and the Chebyshev coefficients for the inner solve:
// [a, b] = [theta_min, 1.02 theta_max] of the Ritz values (modes below a still
// converge; the bound above keeps every mode in (0, a + b)).
void chebyshev_setup(mot_ctx* c) {
    const long long n3 = 3 * c->M;
    const int nb = 256;
    double *v0 = nullptr, *v1 = nullptr, *w = nullptr, *part = nullptr;
    MOT_CUDA_TRY(cudaMalloc(&v0, sizeof(double) * n3));
    MOT_CUDA_TRY(cudaMalloc(&v1, sizeof(double) * n3));
    MOT_CUDA_TRY(cudaMalloc(&w, sizeof(double) * n3));
    MOT_CUDA_TRY(cudaMalloc(&part, sizeof(double) * nb));
    std::vector<double> al, be;
    try {
        std::vector<double> h(n3, 0.0), act(c->nact);
        std::vector<int> ai(c->nact);
        MOT_CUDA_TRY(cudaMemcpy(ai.data(), c->active, sizeof(int) * c->nact, cudaMemcpyDeviceToHost));
        unsigned long long st = 240703323ULL;
        double nrm = 0.0;
        for (long long i = 0; i < c->nact; ++i)
            for (int k = 0; k < 3; ++k) {
                st = st * 6364136223846793005ULL + 1442695040888963407ULL;
                const double r = (double)(st >> 11) / 9007199254740992.0 - 0.5;
                h[k * c->M + ai[i]] = r;
                nrm += r * r;
            }
        nrm = std::sqrt(nrm);
        for (double& x : h) x /= nrm;
        MOT_CUDA_TRY(cudaMemcpy(v1, h.data(), sizeof(double) * n3, cudaMemcpyHostToDevice));
        MOT_CUDA_TRY(cudaMemset(v0, 0, sizeof(double) * n3));
        CGArgs a{};
        a.M = c->M; a.act = c->active; a.nmask = c->nmask; a.nact = c->nact; a.diag = c->cg_diag;
        for (int e = 0; e < 27; ++e) a.noff[e] = c->noff[e];
        auto dot = [&](const double* x, const double* y) {
            k_dot<<<nb, NT, 0, c->stream>>>(x, y, n3, part);
            MOT_LAUNCH_CHECK();
            std::vector<double> hp(nb);
            MOT_CUDA_TRY(cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                                         c->stream));
            MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
            double s = 0.0;
            for (double x : hp) s += x;
            return s;
        };
        double beta = 0.0;
        const int blocks = (int)((n3 + NT - 1) / NT);
        for (int j = 0; j < 40; ++j) {
            MOT_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(double) * n3, c->stream));
            k_apply64<<<(int)((c->nact + NT - 1) / NT), NT, 0, c->stream>>>(a, v1, w);
            MOT_LAUNCH_CHECK();
            const double alpha = dot(w, v1);
            k_axpy2<<<blocks, NT, 0, c->stream>>>(w, v1, alpha, v0, beta, n3);
            MOT_LAUNCH_CHECK();
            al.push_back(alpha);
            be.push_back(beta);
            beta = std::sqrt(std::max(dot(w, w), 0.0));
            if (!(beta > 1e-14)) break;
            k_scale<<<blocks, NT, 0, c->stream>>>(w, 1.0 / beta, n3);
            MOT_LAUNCH_CHECK();
            std::swap(v0, v1);
            std::swap(v1, w);
        }
    } catch (...) {
        cudaFree(v0); cudaFree(v1); cudaFree(w); cudaFree(part);
        throw;
    }
    cudaFree(v0); cudaFree(v1); cudaFree(w); cudaFree(part);
    double lo = 1e300, hi = -1e300;
    for (size_t i = 0; i < al.size(); ++i) {
        const double r = std::fabs(al[i]) + (i ? std::fabs(be[i]) : 0.0) +
                         (i + 1 < al.size() ? std::fabs(be[i + 1]) : 0.0);
        lo = std::min(lo, al[i] - r);
        hi = std::max(hi, al[i] + r);
    }
    const int k = (int)al.size();
    const double tmin = tridiag_eig(al, be, 0, lo, hi);
    const double tmax = tridiag_eig(al, be, k - 1, lo, hi);
    // tmax == tmin when A is a multiple of the identity (a single voxel: G_0(0) is
    // isotropic); the interval [tmin, 1.02 tmax] below is still non-empty
    if (!(tmin > 0.0) || !(tmax >= tmin))
        throw MotError{MOT_ERR_ARG, "diag(1/chi) Z_0 is not positive definite on this grid"};
    const double A = tmin, B = 1.02 * tmax;
    c->cheb_lmin = A;
    c->cheb_lmax = B;
    const double theta = 0.5 * (B + A), delta = 0.5 * (B - A), sigma = theta / delta;
    const double kap = B / A;
    const double rate = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
    int nk = (int)std::ceil(std::log(5e-6) / std::log(rate));
    nk = std::max(4, std::min(nk, MAXCHEB));
    c->cheb_n = nk;
    c->cheb_log_rate = std::log(rate);
    c->cheb_inv_theta = (float)(1.0 / theta);
    double rho = 1.0 / sigma;
    for (int i = 0; i < nk; ++i) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        c->cheb_c1[i] = (float)(rn * rho);
        c->cheb_c2[i] = (float)(2.0 * rn / delta);
        rho = rn;
    }
}

template <typename R>
void epilogue(mot_ctx* c, int n, const double* En, cudaStream_t s) {
    const long long tot = c->M;
    k_epilogue<R><<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(
        c->M, c->vfac, En, hbuf<R>(c).hist_spatial, c->J, (int)slot_index(n, c->jring), c->jring,
        taps_of(c), c->rhs);
    MOT_LAUNCH_CHECK();
}

CGArgs make_cg_args(mot_ctx* c, int n, double* norm2_out) {
    CGArgs a;
    a.M = c->M;
    for (int e = 0; e < 27; ++e) a.noff[e] = c->noff[e];
    a.act = c->active;
    a.nmask = c->nmask;
    a.nact = c->nact;
    a.U = c->U; a.V = c->V; a.W = c->W;
    a.tiles = c->tiles;
    a.ntiles = c->ntiles;
    a.x = c->J + slot_index(n, c->jring) * 3 * c->M;
    a.b = c->rhs;
    a.diag32 = c->diag32;
    a.diag = c->cg_diag;
    a.chi = c->chi;
    a.r64 = c->cg_r;
    a.r = reinterpret_cast<float4*>(c->cg32);
    a.p = a.r + c->M;
    a.q = a.r + 2 * c->M;
    a.e = a.r + 3 * c->M;
    a.xh = a.xl = a.bh = a.bl = nullptr;
    a.diag_lo = nullptr;
    if (c->cg_df) {
        float4* d4 = reinterpret_cast<float4*>(c->cg_df);
        a.xh = d4;
        a.xl = d4 + c->M;
        a.bh = d4 + 2 * c->M;
        a.bl = d4 + 3 * c->M;
        a.diag_lo = c->cg_df + 16 * c->M;
    }
    a.red = c->red;
    a.tol2 = c->tol * c->tol;
    a.inv_theta = c->cheb_inv_theta;
    a.n_cheb = c->cheb_n;
    a.log_rate = c->cheb_log_rate;
    for (int k = 0; k < MAXCHEB; ++k) {
        a.c1[k] = k < c->cheb_n ? c->cheb_c1[k] : 0.f;
        a.c2[k] = k < c->cheb_n ? c->cheb_c2[k] : 0.f;
    }
    a.max_iter = c->max_iter;
    a.max_outer = 12;
    a.step = n;
    a.status = c->dstatus;
    a.bar = reinterpret_cast<unsigned*>(c->dstatus + 4);
    a.bar_budget = c->bar_budget;
    a.norm2 = norm2_out;
    return a;
}

void launch_cg(mot_ctx* c, void** args, cudaStream_t s) {
    void* k = c->precision == MOT_FP64 ? (void*)k_cg<false> : (void*)k_cg<true>;
    MOT_CUDA_TRY(cudaLaunchCooperativeKernel(k, c->cg_blocks, NT, args, 0, s));
}

// rhs + CG for step n; ||J_n||^2 into norm2_out (device), J_n in ring slot n
void solve_step(mot_ctx* c, int n, const double* En, double* norm2_out, cudaStream_t s) {
    if (c->precision == MOT_FP64) epilogue<double>(c, n, En, s);
    else epilogue<float>(c, n, En, s);
    CGArgs a = make_cg_args(c, n, norm2_out);
    void* args[] = {&a};
    launch_cg(c, args, s);
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
            taps_of(c), out_dev);
    else
        k_history_out<float><<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(
            c->M, c->eps, c->chi, c->h32.hist_spatial, c->J, (int)slot_index(n, c->jring), c->jring,
            taps_of(c), out_dev);
    MOT_LAUNCH_CHECK();
}

// one adjoint step: tau = adjoint time (ring index), n = N + 1 - tau (forward time)
void adjoint_step(mot_ctx* c, int tau, int n, const double* g_aos, const double* J_aos,
                  int j_first, double* grad_chi, double* lam_out, double* norm2_out,
                  cudaStream_t s) {
    const long long tot = 3 * c->M;
    const int s0 = (int)slot_index(tau, c->jring);
    if (c->precision == MOT_FP64)
        k_epilogue_adj<double><<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(
            c->M, c->vfac, g_aos, c->h64.hist_spatial, c->J, s0, c->jring, taps_of(c), c->rhs);
    else
        k_epilogue_adj<float><<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(
            c->M, c->vfac, g_aos, c->h32.hist_spatial, c->J, s0, c->jring, taps_of(c), c->rhs);
    MOT_LAUNCH_CHECK();
    CGArgs a = make_cg_args(c, tau, norm2_out);
    void* args[] = {&a};
    launch_cg(c, args, s);
    double* mu = c->J + (long long)s0 * 3 * c->M;
    k_adj_vacuum<<<(int)((c->M + NT - 1) / NT), NT, 0, s>>>(c->M, c->U, c->V, c->W, c->vfac, mu,
                                                           c->rhs, c->cg_q);
    MOT_LAUNCH_CHECK();
    k_adj_post<<<(int)((c->M + NT - 1) / NT), NT, 0, s>>>(c->M, c->vfac, mu, c->cg_q, J_aos,
                                                         j_first, n, taps_of(c), grad_chi,
                                                         lam_out);
    MOT_LAUNCH_CHECK();
    c->stats.launches += 4;
}

void write_aos(mot_ctx* c, int n, double* out_dev, cudaStream_t s) {
    const long long tot = 3 * c->M;
    k_to_aos<<<(int)((tot + NT - 1) / NT), NT, 0, s>>>(c->J + slot_index(n, c->jring) * 3 * c->M,
                                                       c->M, out_dev);
    MOT_LAUNCH_CHECK();
}

}  // namespace mot

extern "C" mot_status mot_barrier_check(int n_blocks, int rounds, int absent, double budget_s,
                                        int* passed, int* timeout_round) {
    if (!passed || !timeout_round || rounds < 1 || rounds > (1 << 20) || absent < -1 ||
        absent >= n_blocks || !(budget_s > 0.0 && budget_s <= 10.0))
        return MOT_ERR_ARG;
    int dev = 0, nsm = 0, per_sm = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_check, NT, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return MOT_ERR_CUDA;
    }
    if (n_blocks < 1 || n_blocks > per_sm * nsm) return MOT_ERR_ARG;   // must be co-resident
    int* w = nullptr;
    if (cudaMalloc(&w, sizeof(int) * 8) != cudaSuccess) {
        cudaGetLastError();
        return MOT_ERR_OOM;
    }
    long long budget = (long long)(budget_s * 1e3 * std::max(khz, 1000000));
    void* args[] = {&w, &budget, &rounds, &absent};
    int h[8] = {0};
    cudaError_t e = cudaMemset(w, 0, sizeof(int) * 8);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((void*)k_barrier_check, n_blocks, NT, args, 0, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(h, w, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(w);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MOT_ERR_CUDA;
    }
    *passed = h[7];
    *timeout_round = h[2];
    return (h[1] & 4) ? MOT_ERR_TIMEOUT : MOT_OK;
}

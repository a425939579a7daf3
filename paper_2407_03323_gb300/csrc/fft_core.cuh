// Shared-memory batched FFT core (mixed-radix Stockham, radices 2, 3, 4, 5, 7), used by
// the spatial FFT passes and the temporal block products.  A tile of TB lines of
// length P is stored as buf[j * ld + t] (ld >= TB); every thread of the CTA takes
// butterflies of every line; tw holds exp(-2 pi i k / P), k < P.
#pragma once

#include "mot_internal.cuh"

#include <type_traits>

namespace mot_fft {

// compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1
template <int B, int E> struct Unroll1 {
    template <typename F> __host__ __device__ __forceinline__ static void run(F&& f) {
        f(std::integral_constant<int, B>());
        Unroll1<B + 1, E>::run(f);
    }
};
template <int E> struct Unroll1<E, E> {
    template <typename F> __host__ __device__ __forceinline__ static void run(F&&) {}
};

// Twiddles known at compile time: cos and sin of 2 pi k / n by the Taylor series of
// sin and cos on [0, pi/4], after reducing the angle with the quadrant and octant
// symmetries in exact integer arithmetic.  Evaluated only by the compiler (constexpr
// initialisers), so butterflies with compile-time indices multiply by literal constants.
struct CTw { double re, im; };
__host__ __device__ constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int i = 1; i < 14; ++i) {
        term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 14; ++i) {
        term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        sum += term;
    }
    return sum;
}
// exp(-2 pi i k / n), 0 <= k < n
__host__ __device__ constexpr CTw root_of_unity(int k, int n) {
    constexpr double pi = 3.141592653589793238462643383279502884;
    const int q = (4 * k) / n;               // quadrant of 2 pi k / n
    const int r = 4 * k - q * n;             // remainder angle = (pi / 2) r / n, r in [0, n)
    const bool hi = 2 * r > n;               // beyond pi / 4: use the complement
    const double phi = (pi / 2.0) * (double)(hi ? n - r : r) / (double)n;
    const double c0 = hi ? taylor_sin(phi) : taylor_cos(phi);
    const double s0 = hi ? taylor_cos(phi) : taylor_sin(phi);
    // angle = q pi/2 + (pi/2) r / n ; (cos, sin) of it
    const double ca = q == 0 ? c0 : (q == 1 ? -s0 : (q == 2 ? -c0 : s0));
    const double sa = q == 0 ? s0 : (q == 1 ? c0 : (q == 2 ? -s0 : -c0));
    return CTw{ca, -sa};
}
static_assert(root_of_unity(0, 8).re == 1.0 && root_of_unity(2, 8).im == -1.0, "twiddle");
static_assert(root_of_unity(4, 8).re == -1.0 && root_of_unity(6, 8).im == 1.0, "twiddle");
static_assert(root_of_unity(1, 6).re - 0.5 < 1e-16 && 0.5 - root_of_unity(1, 6).re < 1e-16,
              "twiddle");
static_assert(root_of_unity(1, 8).re - 0.70710678118654752 < 2e-16 &&
              0.70710678118654752 - root_of_unity(1, 8).re < 2e-16, "twiddle");

// v * W_N^K for compile-time K, N; DIR = -1 forward (W = exp(-2 pi i / N)), +1 inverse
template <int K, int N, int DIR, typename C>
__host__ __device__ __forceinline__ C twiddle_c(C v) {
    typedef decltype(v.x) R;
    if constexpr (K == 0) {
        return v;
    } else if constexpr (4 * K == N) {        // -i (forward) / +i (inverse)
        C o;
        if (DIR < 0) { o.x = v.y; o.y = -v.x; } else { o.x = -v.y; o.y = v.x; }
        return o;
    } else {
        constexpr CTw w = root_of_unity(K, N);
        constexpr double wim = DIR < 0 ? w.im : -w.im;
        constexpr R wr = (R)w.re;
        constexpr R wi = (R)wim;
        C o;
        if constexpr (std::is_same<R, float>::value) {
            // FP32: the constant as a float pair hi + lo, so that the rounding of the
            // twiddle itself (a systematic change of the transform) drops to ~2^-48
            constexpr float wrl = (float)(w.re - (double)wr), wil = (float)(wim - (double)wi);
            const float tx = v.x * wrl - v.y * wil, ty = v.x * wil + v.y * wrl;
            o.x = fmaf(v.x, wr, fmaf(-v.y, wi, tx));
            o.y = fmaf(v.x, wi, fmaf(v.y, wr, ty));
        } else {
            o.x = v.x * wr - v.y * wi;
            o.y = v.x * wi + v.y * wr;
        }
        return o;
    }
}

// A += s cos(2 pi K / N), B += d sin(2 pi K / N) (odd radices, compile-time
// constants); in FP32 each constant is applied as a float pair hi + lo (see twiddle_c)
template <typename Rl, int K, int N, typename C>
__host__ __device__ __forceinline__ void odd_radix_terms(const C& s, const C& d, C& A, C& B) {
    constexpr CTw w = root_of_unity(K, N);   // cos - i sin
    constexpr double CS = w.re, SN = -w.im;
    constexpr Rl cs = (Rl)CS, sn = (Rl)SN;
    if constexpr (std::is_same<Rl, float>::value) {
        constexpr float csl = (float)(CS - (double)cs), snl = (float)(SN - (double)sn);
        A.x = fmaf(s.x, cs, fmaf(s.x, csl, A.x));
        A.y = fmaf(s.y, cs, fmaf(s.y, csl, A.y));
        B.x = fmaf(d.x, sn, fmaf(d.x, snl, B.x));
        B.y = fmaf(d.y, sn, fmaf(d.y, snl, B.y));
    } else {
        A.x += s.x * cs;
        A.y += s.y * cs;
        B.x += d.x * sn;
        B.y += d.y * sn;
    }
}

// In-register DFT of N = 2^a 3^b 5^c 7^d points with compile-time structure:
// X[k] = sum_n x[n] W_N^{nk}, W_N = exp(-2 pi i / N) (DIR = -1) or its conjugate
// (DIR = +1); natural order in and out.  Composite N by decimation in time with the
// smallest factor R first: with n = r + R m and k = k1 + M q (M = N / R),
//   X[k1 + M q] = sum_r W_R^{r q} (W_N^{r k1} sum_m x[r + R m] W_M^{m k1}).
// Odd primes use the symmetric form out[q] = x0 + sum_r (s_r cos - / + i d_r sin)
// with s_r = x_r + x_{R-r}, d_r = x_r - x_{R-r}.
constexpr int smallest_factor(int n) {
    return n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : (n % 5 == 0 ? 5 : 7));
}

template <int N, int DIR, typename C>
__host__ __device__ __forceinline__ void dft_ct(C* x) {
    typedef decltype(x[0].x) Rl;
    if constexpr (N == 1) {
        return;
    } else if constexpr (N == 2) {
        const C a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    } else if constexpr (N == 3 || N == 5 || N == 7) {
        constexpr int H = (N - 1) / 2;
        C s[H], d[H];
        const C v0 = x[0];
        C sum = v0;
        Unroll1<1, H + 1>::run([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            s[r - 1] = cadd(x[r], x[N - r]);
            d[r - 1] = csub(x[r], x[N - r]);
            sum = cadd(sum, s[r - 1]);
        });
        Unroll1<1, H + 1>::run([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            C A = v0, B;
            B.x = 0; B.y = 0;
            Unroll1<1, H + 1>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                odd_radix_terms<Rl, (q * r) % N, N>(s[r - 1], d[r - 1], A, B);
            });
            C mB;   // -i B
            mB.x = B.y; mB.y = -B.x;
            if constexpr (DIR < 0) {
                x[q] = cadd(A, mB);
                x[N - q] = csub(A, mB);
            } else {
                x[q] = csub(A, mB);
                x[N - q] = cadd(A, mB);
            }
        });
        x[0] = sum;
    } else {
        constexpr int R = smallest_factor(N), M = N / R;
        C sub[R][M];
        Unroll1<0, R>::run([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            Unroll1<0, M>::run([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                sub[r][m] = x[r + R * m];
            });
            dft_ct<M, DIR>(sub[r]);
        });
        Unroll1<0, M>::run([&](auto kc) {
            constexpr int k1 = decltype(kc)::value;
            C v[R];
            Unroll1<0, R>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                v[r] = twiddle_c<(r * k1) % N, N, DIR>(sub[r][k1]);
            });
            dft_ct<R, DIR>(v);
            Unroll1<0, R>::run([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                x[k1 + M * q] = v[q];
            });
        });
    }
}

// Twiddle tables: W_P^m = exp(-2 pi i m / P), m < P; the FP32 table holds a second
// block of P entries, the low parts (W - hi rounded to FP32), so that it has
// tw_entries(P) = 2P entries.
template <typename C> __host__ __device__ constexpr int tw_entries(int P) {
    return std::is_same<C, float2>::value ? 2 * P : P;
}
// v * W(m) for dir = -1 (forward), v * conj W(m) for dir = +1, from a table of P
// (FP64) or 2P (FP32: hi and lo parts, the twiddle applied as their sum) entries
__device__ __forceinline__ double2 twmul_tab(const double2* tw, int m, int P, int dir, double2 v) {
    double2 w = tw[m];
    if (dir > 0) w.y = -w.y;
    return cmul(v, w);
}
__device__ __forceinline__ float2 twmul_tab(const float2* tw, int m, int P, int dir, float2 v) {
    float2 h = tw[m], l = tw[P + m];
    if (dir > 0) { h.y = -h.y; l.y = -l.y; }
    const float tx = v.x * l.x - v.y * l.y, ty = v.x * l.y + v.y * l.x;
    float2 o;
    o.x = fmaf(v.x, h.x, fmaf(-v.y, h.y, tx));
    o.y = fmaf(v.x, h.y, fmaf(v.y, h.x, ty));
    return o;
}

template <typename C, int R>
__device__ __forceinline__ void dft_small(C* v, const C* tw, int P, int dir) {
    if constexpr (R == 2) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        C b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
        // -i * dir' : forward multiplies b1 by -i, inverse by +i
        C jb1;
        if (dir < 0) { jb1.x = b1.y; jb1.y = -b1.x; } else { jb1.x = -b1.y; jb1.y = b1.x; }
        v[0] = cadd(a0, b0);
        v[2] = csub(a0, b0);
        v[1] = cadd(a1, jb1);
        v[3] = csub(a1, jb1);
    } else {
        // odd radix: out[q] = v0 + sum_r (s_r cos(2 pi q r/R) -/+ i d_r sin(2 pi q r/R)),
        // with the cosines and sines as compile-time constants
        typedef decltype(v[0].x) Rl;
        constexpr int H = (R - 1) / 2;
        C s[H], d[H];
        const C v0 = v[0];
        C sum = v0;
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            s[r - 1] = cadd(v[r], v[R - r]);
            d[r - 1] = csub(v[r], v[R - r]);
            sum = cadd(sum, s[r - 1]);
        }
        Unroll1<1, H + 1>::run([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            C A = v0, B;
            B.x = 0; B.y = 0;
            Unroll1<1, H + 1>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                odd_radix_terms<Rl, (q * r) % R, R>(s[r - 1], d[r - 1], A, B);
            });
            // forward: out[q] = A - i B, out[R-q] = A + i B ; inverse: swapped
            C mB;   // -i B
            mB.x = B.y; mB.y = -B.x;
            if (dir < 0) {
                v[q] = cadd(A, mB);
                v[R - q] = csub(A, mB);
            } else {
                v[q] = csub(A, mB);
                v[R - q] = cadd(A, mB);
            }
        });
        v[0] = sum;
    }
}

// one Stockham stage of radix R over TB lines (TB known at compile time); Ns is the
// product of the earlier radices; j / Ns is taken as trunc((j + 1/2) / Ns) in FP32,
// exact for j < 2^20
template <typename C, int R, int TB>
__device__ __forceinline__ void stage(const C* __restrict__ x, C* __restrict__ y, int P, int Ns,
                                      int ld, const C* tw, int dir) {
    const int nb = P / R;
    const int items = nb * TB;
    const int tstep = P / (Ns * R);
    const float inv_ns = 1.0f / (float)Ns;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int t = it % TB, j = it / TB;
        const int jq = __float2int_rz(((float)j + 0.5f) * inv_ns);
        const int k = j - jq * Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[(j + r * nb) * ld + t];
        if (Ns > 1) {
            const int kt = k * tstep;      // r * kt < P
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = twmul_tab(tw, r * kt, P, dir, v[r]);
        }
        dft_small<C, R>(v, tw, P, dir);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) y[(base + r * Ns) * ld + t] = v[r];
    }
}

// runs all stages over TB lines of length P; returns the buffer holding the result
template <typename C, int TB>
__device__ C* fft_tile(C* b0, C* b1, int P, const int* rad, int nrad, int ld, const C* tw,
                       int dir) {
    int Ns = 1;
    C* x = b0;
    C* y = b1;
    for (int s = 0; s < nrad; ++s) {
        const int R = rad[s];
        switch (R) {
            case 2: stage<C, 2, TB>(x, y, P, Ns, ld, tw, dir); break;
            case 3: stage<C, 3, TB>(x, y, P, Ns, ld, tw, dir); break;
            case 4: stage<C, 4, TB>(x, y, P, Ns, ld, tw, dir); break;
            case 5: stage<C, 5, TB>(x, y, P, Ns, ld, tw, dir); break;
            case 7: stage<C, 7, TB>(x, y, P, Ns, ld, tw, dir); break;
        }
        __syncthreads();
        Ns *= R;
        C* tmp = x; x = y; y = tmp;
    }
    return x;
}

struct RadixList {
    int P;
    int n;
    int r[16];
};

template <typename C>
__device__ __forceinline__ void load_tw(C* stw, const C* tw, int P) {
    for (int i = threadIdx.x; i < tw_entries<C>(P); i += blockDim.x) stw[i] = tw[i];
}

// Asynchronous global -> shared copy of one complex value (8 or 16 bytes); with
// valid = false nothing is read and the destination is zero-filled.  A tile's copies
// are all issued before one wait, so their memory latencies overlap.
template <typename C>
__device__ __forceinline__ void cp_async_c(C* dst, const C* src, bool valid = true) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(C) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                     "r"(valid ? 8 : 0));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
                     "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit_wait() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}


}  // namespace mot_fft

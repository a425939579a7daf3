// Interaction-element quadrature on the GPU in FP64 (Eq. Z with S of Eq. TDJVIE).
//
// With h = c dt = 1 and C_d(x) = L(x-dx) L(y-dy) L(z-dz) the autocorrelation of two
// unit voxels (L the unit hat), the elements are (with the lag-l time dependence of
// the retarded potential (Sec. 2.1) under the quadratic-spline basis, the curl-curl of
// the field operator written as grad div minus a second time derivative, and the grad
// div moved onto C_d by parts, so that it acts as a double surface integral):
//   K^vol_l(d)      = int C_d(x) T''(l - r) / (4 pi r) dx
//   K^face_l^ab(d)  = int (d_a d_b C_d)(x) T(l - r) / (4 pi r) dx
//   G_l^ab(d)       = K^face_l^ab(d) - delta_ab K^vol_l(d)
// T is the quadratic B-spline on (-1, 2) (Sec. 2.3).  All weights are separable, so in
// cylindrical coordinates about one axis  int w f(r) = int_0^inf s A(s) H(s) ds  with
// A the integral of the in-plane weight over the circle of radius s (closed form per
// arc) and H the axial integral of w_z f (Gauss-Legendre per piece between cell edges
// and shell crossings r = integer; closed form in the shell r < 1).  The s-integral
// is split at every radius where A or H changes form and each piece uses a
// Gauss-Legendre rule after the sigmoidal map u -> u^p / (u^p + (1-u)^p).
//
// One warp per (sorted offset a >= b >= c, cylinder axis); the three axis passes of
// an offset give K^vol and all six K^face components; cubic symmetry maps the sorted
// offsets onto the octant.
#include "mot_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int NS_MAIN = 32;   // nodes per s-interval, p = 2
constexpr int NS_ORIG = 48;   // nodes on an interval that starts at s = 0, p = 3
constexpr int NZ = 16;        // Gauss-Legendre nodes per z piece
constexpr int MAXBP = 96;
constexpr int MAXZC = 32;
constexpr int WARPS_PER_BLOCK = 4;
constexpr double FOURPI = 12.566370614359172953850573533118;

__constant__ double c_sm_t[NS_MAIN], c_sm_w[NS_MAIN];
__constant__ double c_so_t[NS_ORIG], c_so_w[NS_ORIG];
__constant__ double c_gz_x[NZ], c_gz_w[NZ];

// -------------------------------------------------------------- host: Gauss rules
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846264338327950288;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// nodes t in (0,1) and weights of the sigmoidal rule of order p built on n-point GL
void sigmoid_rule(int n, int p, std::vector<double>& t, std::vector<double>& w) {
    std::vector<double> x, g;
    gauss_legendre(n, x, g);
    t.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double u = 0.5 * (x[i] + 1.0), v = 1.0 - u;
        double up = std::pow(u, p), vp = std::pow(v, p);
        double den = up + vp;
        t[i] = up / den;
        w[i] = 0.5 * g[i] * p * std::pow(u, p - 1) * std::pow(v, p - 1) / (den * den);
    }
}

// -------------------------------------------------------------- device helpers
struct Cell {
    double x0, x1, y0, y1, wx0, sx, wy0, sy;
};

// pieces of L(x - d) (deriv 0) or L'(x - d) (deriv 1), reflected into x >= 0:
// (lo, hi, value at lo, slope)
__device__ inline void hat_piece(double d, int which, int deriv, double& lo, double& hi,
                                 double& v0, double& sl) {
    if (which == 0) {
        lo = d - 1.0; hi = d;
        v0 = deriv ? 1.0 : 0.0; sl = deriv ? 0.0 : 1.0;
    } else {
        lo = d; hi = d + 1.0;
        v0 = deriv ? -1.0 : 1.0; sl = deriv ? 0.0 : -1.0;
    }
    if (hi <= 0.0) {  // only the piece [-1, 0] of d = 0: mirror x -> -x
        double nlo = -hi, nhi = -lo;
        // value at the new lower end (old upper end) and mirrored slope
        double vnew = v0 + sl * (hi - lo);
        lo = nlo; hi = nhi; v0 = vnew; sl = -sl;
    }
}

__device__ inline Cell make_cell(double dp, double dq, int i, int j, int deriv) {
    Cell c;
    hat_piece(dp, i, deriv, c.x0, c.x1, c.wx0, c.sx);
    hat_piece(dq, j, deriv, c.y0, c.y1, c.wy0, c.sy);
    return c;
}

// int_{-h}^{h} (cos t - 1) dt, sin^2 t dt, (cos t - 1)^2 dt without cancellation
__device__ inline void arc_moments(double h, double& Ic, double& Iss, double& Icc) {
    if (h < 0.5) {
        double h2 = h * h, pw = h * h2;   // h^(2k+1), k = 1
        double fact = 6.0;                // (2k+1)!
        double four = 4.0;                // 2^(2k)
        Ic = 0.0; Iss = 0.0; Icc = 0.0;
        double sgn = -1.0;                // (-1)^k
        for (int k = 1; k <= 10; ++k) {
            double term = pw / fact;
            Ic += 2.0 * sgn * term;
            Iss += -sgn * four * term;
            Icc += sgn * (four - 4.0) * term;
            pw *= h2;
            fact *= (2.0 * k + 2.0) * (2.0 * k + 3.0);
            four *= 4.0;
            sgn = -sgn;
        }
    } else {
        double sh, ch;
        sincos(h, &sh, &ch);
        Ic = 2.0 * sh - 2.0 * h;
        Iss = h - sh * ch;
        Icc = 3.0 * h + sh * ch - 4.0 * sh;
    }
}

// integral over the circle of radius s of the cell weight (first-quadrant cell)
__device__ inline double arc_cell(double s, const Cell& c) {
    if (!(c.x0 < s && c.y0 < s)) return 0.0;
    double s2 = s * s;
    double Xa, Ya, Xb, Yb;
    {   // lower end: larger angle of {leave x <= x1, enter y >= y0}
        double xa1 = c.x1 < s ? c.x1 : s;
        double ya1 = c.x1 < s ? sqrt(fmax(s2 - c.x1 * c.x1, 0.0)) : 0.0;
        double xa2 = sqrt(fmax(s2 - c.y0 * c.y0, 0.0));
        double ya2 = c.y0;
        if (ya2 > ya1) { Xa = xa2; Ya = ya2; } else { Xa = xa1; Ya = ya1; }
    }
    {   // upper end: smaller angle of {leave x >= x0, leave y <= y1}
        double xb1 = c.x0, yb1 = sqrt(fmax(s2 - c.x0 * c.x0, 0.0));
        double xb2 = c.y1 < s ? sqrt(fmax(s2 - c.y1 * c.y1, 0.0)) : 0.0;
        double yb2 = c.y1 < s ? c.y1 : s;
        if (yb2 < yb1) { Xb = xb2; Yb = yb2; } else { Xb = xb1; Yb = yb1; }
    }
    if (!(Yb > Ya)) return 0.0;
    double pa = atan2(Ya, Xa), pb = atan2(Yb, Xb);
    double h = 0.5 * (pb - pa);
    if (h <= 0.0) return 0.0;
    double sm, cm;
    sincos(0.5 * (pa + pb), &sm, &cm);
    double Xm = s * cm, Ym = s * sm;
    double Ax = c.wx0 + c.sx * (Xm - c.x0);
    double Ay = c.wy0 + c.sy * (Ym - c.y0);
    double Ic, Iss, Icc;
    arc_moments(h, Ic, Iss, Icc);
    return 2.0 * h * Ax * Ay + (Ax * c.sy * Ym + Ay * c.sx * Xm) * Ic +
           c.sx * c.sy * Xm * Ym * (Icc - Iss);
}

__device__ inline void add3(double* acc, int idx, double v0, double v1, double v2,
                            int* bad) {
    if (idx < 0 || idx + 2 >= mot::WIN) { *bad = 1; return; }
    acc[idx] += v0;
    acc[idx + 1] += v1;
    acc[idx + 2] += v2;
}

__device__ inline void sort_small(double* a, int n) {
    for (int i = 1; i < n; ++i) {
        double v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
        a[j + 1] = v;
    }
}

// one axis pass: in-plane offsets (dp, dq), axial dz, lag window starting at l0
__global__ void quad_kernel(const int3* __restrict__ triples, int ntriples,
                            double* __restrict__ out, int* __restrict__ errflag) {
    __shared__ double sbp[WARPS_PER_BLOCK][MAXBP];
    __shared__ int snbp[WARPS_PER_BLOCK];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const long long job = (long long)blockIdx.x * WARPS_PER_BLOCK + wib;
    if (job >= 3LL * ntriples) return;
    const int t = (int)(job / 3), axis = (int)(job % 3);
    const int3 key = triples[t];
    double a = key.x, b = key.y, cc = key.z;
    double dp, dq, dz;
    if (axis == 0) { dp = a; dq = b; dz = cc; }        // axis z: plane (x, y)
    else if (axis == 1) { dp = b; dq = cc; dz = a; }   // axis x: plane (y, z)
    else { dp = cc; dq = a; dz = b; }                  // axis y: plane (z, x)

    const double rmin = sqrt(fmax(a - 1.0, 0.0) * fmax(a - 1.0, 0.0) +
                             fmax(b - 1.0, 0.0) * fmax(b - 1.0, 0.0) +
                             fmax(cc - 1.0, 0.0) * fmax(cc - 1.0, 0.0));
    const int l0 = (int)floor(rmin);
    Cell cL[4], cD[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            cL[2 * i + j] = make_cell(dp, dq, i, j, 0);
            cD[2 * i + j] = make_cell(dp, dq, i, j, 1);
        }
    // the in-plane weight vanishes for s outside [smin, smax]
    double smax = 0.0, smin = 1e300;
    for (int i = 0; i < 4; ++i) {
        smax = fmax(smax, hypot(cL[i].x1, cL[i].y1));
        smin = fmin(smin, hypot(cL[i].x0, cL[i].y0));
    }
    const double zk0 = dz - 1.0, zk1 = dz, zk2 = dz + 1.0;
    const double zmax = fmax(fabs(zk0), fabs(zk2));
    const double rmax = hypot(smax, zmax);
    const int J = (int)floor(rmax) + 1;
    const int J0 = max((int)floor(rmin), 1);

    if (lane == 0) {
        double* bp = sbp[wib];
        int n = 0;
        bp[n++] = smin;
        bp[n++] = smax;
        for (int i = 0; i < 4; ++i) {
            const Cell& c = cL[i];
            bp[n++] = c.x0; bp[n++] = c.x1; bp[n++] = c.y0; bp[n++] = c.y1;
            bp[n++] = hypot(c.x0, c.y0); bp[n++] = hypot(c.x0, c.y1);
            bp[n++] = hypot(c.x1, c.y0); bp[n++] = hypot(c.x1, c.y1);
        }
        const double zks[3] = {zk0, zk1, zk2};
        for (int j = J0; j <= J && n < MAXBP - 4; ++j) {
            bp[n++] = (double)j;
            for (int e = 0; e < 3; ++e)
                if (j > fabs(zks[e])) bp[n++] = sqrt((double)j * j - zks[e] * zks[e]);
        }
        for (int i = 0; i < n; ++i) bp[i] = fmin(fmax(bp[i], smin), smax);
        sort_small(bp, n);
        int m = 1;
        for (int i = 1; i < n; ++i)
            if (bp[i] - bp[m - 1] > 1e-14 * fmax(1.0, bp[i])) bp[m++] = bp[i];
        snbp[wib] = m;
    }
    __syncwarp();
    const int nbp = snbp[wib];
    const double* bp = sbp[wib];

    double accV[mot::WIN], accD[mot::WIN], accO[mot::WIN];
    for (int i = 0; i < mot::WIN; ++i) { accV[i] = 0.0; accD[i] = 0.0; accO[i] = 0.0; }
    int bad = 0;

    for (int iv = 0; iv + 1 < nbp; ++iv) {
        const double sa = bp[iv], sb = bp[iv + 1];
        const bool orig = (sa == 0.0);
        const int ns = orig ? NS_ORIG : NS_MAIN;
        for (int node = lane; node < ns; node += 32) {
            const double tt = orig ? c_so_t[node] : c_sm_t[node];
            const double ww = orig ? c_so_w[node] : c_sm_w[node];
            const double s = sa + (sb - sa) * tt;
            const double Ws = (sb - sa) * ww * s;
            double AL = 0.0, AD = 0.0;
            for (int i = 0; i < 4; ++i) { AL += arc_cell(s, cL[i]); AD += arc_cell(s, cD[i]); }
            const double oL = Ws * AL, oD = Ws * AD;
            if (oL == 0.0 && oD == 0.0) continue;
            // diagonal face term: z-weight delta(z-dz+1) - 2 delta(z-dz) + delta(z-dz-1)
            {
                const double zks[3] = {zk0, zk1, zk2};
                const double we[3] = {1.0, -2.0, 1.0};
                for (int e = 0; e < 3; ++e) {
                    const double r = sqrt(s * s + zks[e] * zks[e]);
                    const int j = (int)floor(r);
                    const double sg = r - j;
                    const double base = we[e] * oL / (FOURPI * r);
                    add3(accD, j - l0, base * 0.5 * (1.0 - sg) * (1.0 - sg),
                         base * 0.5 * (1.0 + 2.0 * sg - 2.0 * sg * sg), base * 0.5 * sg * sg,
                         &bad);
                }
            }
            // axial hat weight: pieces between knots and shell crossings
            double zc[MAXZC];
            int nz = 0;
            zc[nz++] = zk0; zc[nz++] = zk1; zc[nz++] = zk2;
            for (int j = J0; j <= J && nz < MAXZC - 2; ++j) {
                if ((double)j > s) {
                    const double q = sqrt(((double)j - s) * ((double)j + s));
                    if (q > zk0 && q < zk2) zc[nz++] = q;
                    if (-q > zk0 && -q < zk2) zc[nz++] = -q;
                }
            }
            sort_small(zc, nz);
            for (int ip = 0; ip + 1 < nz; ++ip) {
                const double z0 = zc[ip], z1 = zc[ip + 1];
                if (!(z1 > z0)) continue;
                const double zm = 0.5 * (z0 + z1), hz = 0.5 * (z1 - z0);
                const bool lower = zm < dz;
                const int j = (int)floor(sqrt(s * s + zm * zm));
                if (j == 0) {
                    // closed form: int (wa + wb z) r^k dz, k = -1, 0, 1
                    const double wa = lower ? 1.0 - dz : 1.0 + dz, wb = lower ? 1.0 : -1.0;
                    const double r0 = sqrt(s * s + z0 * z0), r1 = sqrt(s * s + z1 * z1);
                    const double as0 = asinh(z0 / s), as1 = asinh(z1 / s);
                    const double Im1 = wa * (as1 - as0) + wb * (r1 - r0);
                    const double I0 = wa * (z1 - z0) + wb * 0.5 * (z1 * z1 - z0 * z0);
                    const double I1 = wa * 0.5 * ((z1 * r1 + s * s * as1) - (z0 * r0 + s * s * as0)) +
                                      wb * (r1 * r1 * r1 - r0 * r0 * r0) / 3.0;
                    const double cv = oL / FOURPI;
                    add3(accV, -l0, cv * Im1, -2.0 * cv * Im1, cv * Im1, &bad);
                    const double co = oD / (2.0 * FOURPI);
                    add3(accO, -l0, co * (Im1 - 2.0 * I0 + I1), co * (Im1 + 2.0 * I0 - 2.0 * I1),
                         co * I1, &bad);
                } else {
                    double v0 = 0.0, v1 = 0.0, v2 = 0.0, o0 = 0.0, o1 = 0.0, o2 = 0.0;
                    for (int g = 0; g < NZ; ++g) {
                        const double z = zm + hz * c_gz_x[g];
                        const double wz = hz * c_gz_w[g] * (lower ? (z - zk0) : (zk2 - z));
                        const double r = sqrt(s * s + z * z);
                        const double sg = r - j;
                        const double q = wz / (FOURPI * r);
                        v0 += q;
                        o0 += q * 0.5 * (1.0 - sg) * (1.0 - sg);
                        o1 += q * 0.5 * (1.0 + 2.0 * sg - 2.0 * sg * sg);
                        o2 += q * 0.5 * sg * sg;
                    }
                    v1 = -2.0 * v0;
                    v2 = v0;
                    add3(accV, j - l0, oL * v0, oL * v1, oL * v2, &bad);
                    add3(accO, j - l0, oD * o0, oD * o1, oD * o2, &bad);
                }
            }
        }
    }
    // warp reduction
    for (int i = 0; i < mot::WIN; ++i) {
        for (int o = 16; o > 0; o >>= 1) {
            accV[i] += __shfl_down_sync(0xffffffffu, accV[i], o);
            accD[i] += __shfl_down_sync(0xffffffffu, accD[i], o);
            accO[i] += __shfl_down_sync(0xffffffffu, accO[i], o);
        }
    }
    if (bad) atomicExch(errflag, 1);
    if (lane == 0) {
        double* o = out + ((long long)t * 3 + axis) * 3 * mot::WIN;
        for (int i = 0; i < mot::WIN; ++i) {
            o[i] = accV[i];
            o[mot::WIN + i] = accD[i];
            o[2 * mot::WIN + i] = accO[i];
        }
    }
}

// Rank of a sorted triple a >= b >= c among the triples a grid needs: with the grid's
// sides sorted L1 >= L2 >= L3, exactly those with a < L1, b < L2, c < L3 (the k-th
// largest offset coordinate is below the k-th largest side), enumerated by a, then b,
// then c.  For a given b there are min(b, L3 - 1) + 1 values of c, so the triples with
// first b' < b number g(b) = b (b + 1) / 2 (b <= L3), L3 (L3 + 1) / 2 + (b - L3) L3
// (b > L3); off_a[a] counts the triples with first coordinate below a.
__host__ __device__ inline long long tri_before_b(long long b, long long L3) {
    return b <= L3 ? b * (b + 1) / 2 : L3 * (L3 + 1) / 2 + (b - L3) * L3;
}

// G_l^{ab}(d) = K^face^{ab} - delta_ab K^vol for lags l0 .. l0 + WIN - 1 of the offset
// d >= 0 (componentwise) from the three axis passes `res` of its sorted triple: the face
// matrix of the sorted frame, permuted back to d's axes.  Writes the six components
// (xx, yy, zz, xy, xz, yz) at dst[c * cstride + i * lstride] and returns l0.
__device__ inline int assemble_window(const double* __restrict__ res, const int d[3],
                                      double* __restrict__ dst, long long cstride,
                                      long long lstride) {
    // sort descending with the permutation p: d[i] = key[p[i]]
    int order[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (d[order[j]] > d[order[i]]) { int tmp = order[i]; order[i] = order[j]; order[j] = tmp; }
    int key[3] = {d[order[0]], d[order[1]], d[order[2]]};
    int p[3];
    for (int k = 0; k < 3; ++k) p[order[k]] = k;
    const double* r0 = res;                       // axis z pass
    const double* r1 = res + 3 * mot::WIN;        // axis x pass
    const double* r2 = res + 6 * mot::WIN;        // axis y pass
    // face matrix in the sorted frame
    const double* F[3][3];
    F[2][2] = r0 + mot::WIN; F[0][1] = r0 + 2 * mot::WIN; F[1][0] = F[0][1];
    F[0][0] = r1 + mot::WIN; F[1][2] = r1 + 2 * mot::WIN; F[2][1] = F[1][2];
    F[1][1] = r2 + mot::WIN; F[0][2] = r2 + 2 * mot::WIN; F[2][0] = F[0][2];
    const double* vol = r0;
    const double rmin = sqrt((double)(max(key[0] - 1, 0) * max(key[0] - 1, 0) +
                                      max(key[1] - 1, 0) * max(key[1] - 1, 0) +
                                      max(key[2] - 1, 0) * max(key[2] - 1, 0)));
    const int comp_a[6] = {0, 1, 2, 0, 0, 1}, comp_b[6] = {0, 1, 2, 1, 2, 2};
    for (int cc = 0; cc < 6; ++cc) {
        const int aa = comp_a[cc], bb = comp_b[cc];
        const double* f = F[p[aa]][p[bb]];
        for (int i = 0; i < mot::WIN; ++i)
            dst[cc * cstride + i * lstride] = f[i] - (aa == bb ? vol[i] : 0.0);
    }
    return (int)floor(rmin);
}

// octant assembly: G_l^{ab}(d) = K^face^{ab} - delta_ab K^vol, windowed in lag
__global__ void assemble_kernel(const double* __restrict__ res, int U, int V, int W,
                                const long long* __restrict__ off_a, int L3,
                                int* __restrict__ tab_l0, double* __restrict__ tab) {
    const long long oct = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)U * V * W;
    if (oct >= n) return;
    const int d[3] = {(int)(oct % U), (int)((oct / U) % V), (int)(oct / ((long long)U * V))};
    int key[3] = {d[0], d[1], d[2]};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (key[j] > key[i]) { int tmp = key[i]; key[i] = key[j]; key[j] = tmp; }
    const long long t = off_a[key[0]] + tri_before_b(key[1], L3) + key[2];
    tab_l0[oct] = assemble_window(res + t * 9 * mot::WIN, d, tab + oct * 6 * mot::WIN, mot::WIN, 1);
}

// Probe windows: for probe p (lattice indices, outside the grid or not) and voxel m,
// G_l(r_p - r_m) for lags l0 .. l0 + WIN - 1 with the parity signs of the full offset
// (diagonal components even in every d_i, the (a, b) component odd in d_a and in d_b,
// zero when either is 0).  Layout tab[p][c][i][m] (voxels fastest), l0[p][m].
__global__ void assemble_probe_kernel(const double* __restrict__ res, const int* __restrict__ kidx,
                                      int A, const int3* __restrict__ probes, int np, int U, int V,
                                      int W, int* __restrict__ l0, double* __restrict__ tab) {
    const long long M = (long long)U * V * W;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * np) return;
    const int p = (int)(i / M);
    const long long m = i % M;
    const int3 q = probes[p];
    const int d[3] = {q.x - (int)(m % U), q.y - (int)((m / U) % V), q.z - (int)(m / ((long long)U * V))};
    const int ad[3] = {abs(d[0]), abs(d[1]), abs(d[2])};
    int key[3] = {ad[0], ad[1], ad[2]};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (key[b] > key[a]) { int tmp = key[a]; key[a] = key[b]; key[b] = tmp; }
    const long long t = kidx[((long long)key[0] * (A + 1) + key[1]) * (A + 1) + key[2]];
    double w[6 * mot::WIN];
    const int lo = assemble_window(res + t * 9 * mot::WIN, ad, w, mot::WIN, 1);
    const double sx = (d[0] > 0) - (d[0] < 0), sy = (d[1] > 0) - (d[1] < 0),
                 sz = (d[2] > 0) - (d[2] < 0);
    const double sgn[6] = {1.0, 1.0, 1.0, sx * sy, sx * sz, sy * sz};
    for (int c = 0; c < 6; ++c)
        for (int k = 0; k < mot::WIN; ++k)
            tab[(((long long)p * 6 + c) * mot::WIN + k) * M + m] = w[c * mot::WIN + k] * sgn[c];
    l0[(long long)p * M + m] = lo;
}

}  // namespace

namespace mot {

void probe_windows(mot_ctx* c, int np, const int* probes, double* tab, int* l0) {
    const int N[3] = {c->U, c->V, c->W};
    // largest offset component over all probe-voxel pairs
    int A = 0;
    for (int p = 0; p < np; ++p)
        for (int a = 0; a < 3; ++a) {
            A = std::max(A, std::abs(probes[3 * p + a]));
            A = std::max(A, std::abs(probes[3 * p + a] - (N[a] - 1)));
        }
    if ((long long)(A + 1) * (A + 1) * (A + 1) > (1LL << 28))
        throw MotError{MOT_ERR_ARG, "probes too far from the grid (offset table over 2^28 entries)"};
    const long long A1 = A + 1;
    std::vector<int> kidx((size_t)(A1 * A1 * A1), -1);
    std::vector<int3> tri;
    for (int p = 0; p < np; ++p)
        for (int w = 0; w < c->W; ++w)
            for (int v = 0; v < c->V; ++v)
                for (int u = 0; u < c->U; ++u) {
                    int k[3] = {std::abs(probes[3 * p] - u), std::abs(probes[3 * p + 1] - v),
                                std::abs(probes[3 * p + 2] - w)};
                    std::sort(k, k + 3, [](int x, int y) { return x > y; });
                    int& slot = kidx[(size_t)((k[0] * A1 + k[1]) * A1 + k[2])];
                    if (slot < 0) {
                        slot = (int)tri.size();
                        tri.push_back(make_int3(k[0], k[1], k[2]));
                    }
                }
    double* res = quad_windows(c, tri);
    int* dk = nullptr;
    int3* dp = nullptr;
    try {
        MOT_CUDA_TRY(cudaMalloc(&dk, sizeof(int) * kidx.size()));
        MOT_CUDA_TRY(cudaMalloc(&dp, sizeof(int3) * np));
        MOT_CUDA_TRY(cudaMemcpyAsync(dk, kidx.data(), sizeof(int) * kidx.size(),
                                     cudaMemcpyHostToDevice, c->stream));
        MOT_CUDA_TRY(cudaMemcpyAsync(dp, probes, sizeof(int3) * np, cudaMemcpyHostToDevice,
                                     c->stream));
        const long long tot = c->M * np;
        assemble_probe_kernel<<<(int)((tot + 255) / 256), 256, 0, c->stream>>>(
            res, dk, A, dp, np, c->U, c->V, c->W, l0, tab);
        MOT_LAUNCH_CHECK();
        MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
    } catch (...) {
        cudaFree(res);
        cudaFree(dk);
        cudaFree(dp);
        throw;
    }
    cudaFree(res);
    cudaFree(dk);
    cudaFree(dp);
}


// Element windows of arbitrary sorted triples a >= b >= c >= 0 (the three axis passes,
// [t][3][3][WIN], device memory owned by the caller); the rules are in constant memory
// after compute_table has run on this device.
double* quad_windows(mot_ctx* c, const std::vector<int3>& tri) {
    const int nt = (int)tri.size();
    int3* dtri = nullptr;
    double* dres = nullptr;
    int* derr = nullptr;
    try {
        MOT_CUDA_TRY(cudaMalloc(&dtri, sizeof(int3) * std::max(nt, 1)));
        MOT_CUDA_TRY(cudaMalloc(&dres, sizeof(double) * (size_t)std::max(nt, 1) * 9 * WIN));
        MOT_CUDA_TRY(cudaMalloc(&derr, sizeof(int)));
        MOT_CUDA_TRY(cudaMemsetAsync(derr, 0, sizeof(int), c->stream));
        if (nt > 0) {
            MOT_CUDA_TRY(cudaMemcpyAsync(dtri, tri.data(), sizeof(int3) * nt,
                                         cudaMemcpyHostToDevice, c->stream));
            const long long jobs = 3LL * nt;
            const int blocks = (int)((jobs + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
            quad_kernel<<<blocks, 32 * WARPS_PER_BLOCK, 0, c->stream>>>(dtri, nt, dres, derr);
            MOT_LAUNCH_CHECK();
        }
        int herr = 0;
        MOT_CUDA_TRY(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (herr) throw MotError{MOT_ERR_CUDA, "element quadrature: lag window overflow"};
    } catch (...) {
        cudaFree(dtri);
        cudaFree(dres);
        cudaFree(derr);
        throw;
    }
    cudaFree(dtri);
    cudaFree(derr);
    return dres;
}

void compute_table(mot_ctx* c) {
    {
        std::vector<double> t, w;
        sigmoid_rule(NS_MAIN, 2, t, w);
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_sm_t, t.data(), sizeof(double) * NS_MAIN));
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_sm_w, w.data(), sizeof(double) * NS_MAIN));
        sigmoid_rule(NS_ORIG, 3, t, w);
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_so_t, t.data(), sizeof(double) * NS_ORIG));
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_so_w, w.data(), sizeof(double) * NS_ORIG));
        gauss_legendre(NZ, t, w);
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_gz_x, t.data(), sizeof(double) * NZ));
        MOT_CUDA_TRY(cudaMemcpyToSymbol(c_gz_w, w.data(), sizeof(double) * NZ));
    }
    // the sorted offsets a >= b >= c that occur in this grid (see tri_before_b)
    int L[3] = {c->U, c->V, c->W};
    std::sort(L, L + 3, [](int x, int y) { return x > y; });
    std::vector<int3> tri;
    std::vector<long long> off_a(L[0]);
    for (int a = 0; a < L[0]; ++a) {
        off_a[a] = (long long)tri.size();
        for (int b = 0; b <= std::min(a, L[1] - 1); ++b)
            for (int cc = 0; cc <= std::min(b, L[2] - 1); ++cc) tri.push_back(make_int3(a, b, cc));
    }
    const int nt = (int)tri.size();
    int3* dtri = nullptr;
    double* dres = nullptr;
    int* derr = nullptr;
    long long* doff = nullptr;
    try {
        MOT_CUDA_TRY(cudaMalloc(&doff, sizeof(long long) * L[0]));
        MOT_CUDA_TRY(cudaMemcpyAsync(doff, off_a.data(), sizeof(long long) * L[0],
                                     cudaMemcpyHostToDevice, c->stream));
        MOT_CUDA_TRY(cudaMalloc(&dtri, sizeof(int3) * nt));
        MOT_CUDA_TRY(cudaMalloc(&dres, sizeof(double) * (size_t)nt * 3 * 3 * WIN));
        MOT_CUDA_TRY(cudaMalloc(&derr, sizeof(int)));
        MOT_CUDA_TRY(cudaMemsetAsync(derr, 0, sizeof(int), c->stream));
        MOT_CUDA_TRY(cudaMemcpyAsync(dtri, tri.data(), sizeof(int3) * nt, cudaMemcpyHostToDevice,
                                     c->stream));
        const long long jobs = 3LL * nt;
        const int blocks = (int)((jobs + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
        quad_kernel<<<blocks, 32 * WARPS_PER_BLOCK, 0, c->stream>>>(dtri, nt, dres, derr);
        MOT_LAUNCH_CHECK();
        const long long noff = (long long)c->U * c->V * c->W;
        MOT_CUDA_TRY(cudaMalloc(&c->tab_l0, sizeof(int) * noff));
        MOT_CUDA_TRY(cudaMalloc(&c->tab, sizeof(double) * noff * 6 * WIN));
        assemble_kernel<<<(int)((noff + 255) / 256), 256, 0, c->stream>>>(
            dres, c->U, c->V, c->W, doff, L[2], c->tab_l0, c->tab);
        MOT_LAUNCH_CHECK();
        int herr = 0;
        MOT_CUDA_TRY(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        MOT_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (herr) throw MotError{MOT_ERR_CUDA, "element quadrature: lag window overflow"};
    } catch (...) {
        cudaFree(dtri);
        cudaFree(dres);
        cudaFree(derr);
        cudaFree(doff);
        throw;
    }
    cudaFree(dtri);
    cudaFree(dres);
    cudaFree(derr);
    cudaFree(doff);
}

}  // namespace mot

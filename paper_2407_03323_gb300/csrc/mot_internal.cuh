// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <type_traits>
#include <vector>

#include "mot.h"

// ------------------------------------------------------------------ complex helpers
template <typename R> struct CT;
template <> struct CT<double> { typedef double2 c; };
template <> struct CT<float>  { typedef float2 c; };

__host__ __device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// ------------------------------------------------------------------ status plumbing
struct MotError {
    mot_status st;
    std::string msg;
};

#define MOT_CUDA_TRY(expr)                                                            \
    do {                                                                              \
        cudaError_t e_ = (expr);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            cudaGetLastError(); /* clear a non-sticky error (e.g. a failed malloc) */ \
            char b_[512];                                                             \
            snprintf(b_, sizeof b_, "%s failed at %s:%d: %s", #expr, __FILE__,        \
                     __LINE__, cudaGetErrorString(e_));                               \
            throw MotError{e_ == cudaErrorMemoryAllocation ? MOT_ERR_OOM : MOT_ERR_CUDA, \
                           b_};                                                       \
        }                                                                             \
    } while (0)

#define MOT_LAUNCH_CHECK() MOT_CUDA_TRY(cudaGetLastError())

// ------------------------------------------------------------------ FFT plan
// One axis of length P = product of radices (each 2, 3, 4, 5 or 7), Stockham order.
struct AxisFFT {
    int P = 0;
    int nrad = 0;
    int rad[16] = {0};
    double2* tw64 = nullptr;  // exp(-2 pi i k / P), k < P (device)
    float2* tw32 = nullptr;   // the same rounded to FP32 (k < P), then the low parts
                              // exp(..) - hi rounded to FP32 (P + k): 2P entries
};

// Device-side precision-dependent buffers.
template <typename R> struct HistoryBuffers {
    typedef typename CT<R>::c C;
    C* jhat_ring = nullptr;      // [slots][3][Pw][Pv][Hu]
    R* ghat = nullptr;           // [lags][6][Hw][Hv][Hu] (lag 1 first)
    C* phat = nullptr;           // [3][Pw][Pv][Hu]
    C* tmp1 = nullptr;           // FFT intermediates
    C* tmp2 = nullptr;
    R* hist_spatial = nullptr;   // [3][W][V][U]   (G * J history, spatial)
    // blocked temporal scheme
    C* acc_ring = nullptr;       // per level [S][3][Pw][Pv][Hu] future far-lag sums
    C* level_spec = nullptr;     // per level kernel temporal spectra (octant)
};

struct mot_ctx {
    int U = 0, V = 0, W = 0;
    long long M = 0;
    int ell = 0;
    AxisFFT ax[3];               // x (u), y (v), z (w)
    int Hu = 0, Hv = 0, Hw = 0;  // P_i / 2 + 1
    long long nbins = 0;         // Pw * Pv * Hu
    long long noct = 0;          // Hw * Hv * Hu
    int precision = 0, scheme = 0, block = 0;
    int n_taps = 0;
    std::vector<double> taps;
    double tol = 1e-13;
    int max_iter = 200;
    double growth = 1e12;

    // ring bookkeeping
    int n_done = 0;              // steps marched
    int jring = 0;               // spatial J ring slots
    int hring = 0;               // spectral J ring slots

    // device: geometry and solve
    double* eps = nullptr;
    double* chi = nullptr;
    double* cg_diag = nullptr;   // (T(0)/eps + delta_0)/chi on active voxels, 0 elsewhere
    double* J = nullptr;         // spatial J ring [jring][3][M] (SoA per slot)
    double* rhs = nullptr;       // [3][M]
    double* cg_r = nullptr;
    float* cg_df = nullptr;      // FP32-history: x, b as float pairs ([4][M] float4), diag low parts [M]
    double* cg_q = nullptr;
    float* cg32 = nullptr;       // FP32 inner CG vectors r, p, q, e ([4][M] float4)
    int* active = nullptr;       // voxels with chi > 0
    int* nmask = nullptr;        // per active voxel: in-grid neighbours (27 bits)
    int* tiles = nullptr;        // 8^3 tiles holding active voxels (packed origins)
    int ntiles = 0;
    float* diag32 = nullptr;     // FP32 copy of cg_diag
    double* vfac = nullptr;      // [4][M]: 0.5/eps, 1/chi (0 if chi = 0), 1/(0.5/eps + d0), chi
    long long nact = 0;
    double cheb_lmin = 0.0, cheb_lmax = 0.0;   // spectral bounds of diag(1/chi) Z_0
    int cheb_n = 0;
    double cheb_log_rate = -1.0;
    float cheb_inv_theta = 0.f;
    float cheb_c1[64] = {0}, cheb_c2[64] = {0};
    double* red = nullptr;       // reduction scratch
    int* dstatus = nullptr;      // [0] cg iterations of last step, [1] flags, [2] first bad
                                 // step, [3] total iterations, [4..6] the solve kernel's
                                 // grid barrier (arrivals, generation, abort)
    long long bar_budget = 0;    // longest barrier wait of the solve kernel, SM clock cycles
    double* norms = nullptr;     // per-step ||J_n||^2 of the current call
    int norms_cap = 0;
    double* outbuf = nullptr;    // kOutSlots steps of AoS J for host outputs (a ring)
    // host transfers overlapped with the march: copy streams (device-to-host outputs,
    // host-to-device excitation, so both directions run at once), per-slot events of the
    // output ring (AoS J written / copied out), and per-chunk events of a host
    // excitation being staged
    cudaStream_t cstream = nullptr;
    cudaStream_t hstream = nullptr;
    cudaEvent_t out_ready[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t out_done[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> e_chunk;
    int e_chunk_steps = 0;       // steps per staged chunk; 0: staged synchronously on the stream
    double last_norm = 0.0;
    double peak_norm = 0.0;
    int fail_step = 0;
    int last_iters = 0;
    double stencil[27 * 6];      // G_0(d) for |d_i| <= 1 (host copy)
    int noff[27] = {0};          // voxel-index offset of neighbour e (the 27-point stencil)

    // interaction table (sparse in lag): per octant offset, window of WIN lags
    int* tab_l0 = nullptr;       // [W*V*U]
    double* tab = nullptr;       // [W*V*U][6][WIN]

    // excitation staging
    double* Estage = nullptr;    // [cap][M][3]
    double* pw_tab = nullptr;    // [kPwTable] plane-wave voxel-average table (excitation.cu)
    int E_cap = 0, E_count = 0, E_first = 0;  // steps staged, first staged n

    HistoryBuffers<double> h64;
    HistoryBuffers<float> h32;
    int nlev = 0;                // blocked scheme levels: lags [lev_a, lev_a + lev_S)
    int lev_S[8] = {0};          // level length S (fires every S steps, transform 2S)
    int lev_a[8] = {0};          // its first lag (S for the doubling levels B, 2B, ...)
    int lev_period = 1;          // the longest S: the firing pattern repeats with it
    bool lev_fit = true;         // last level fitted to ell (MOT_HISTORY_BLOCKED)
    long long lev_off[8] = {0};  // offsets of the level spectra
    AxisFFT lev_fft[8];          // temporal FFT plans of length 2S
    long long lev_acc[8] = {0};  // first accumulator slot of each level's ring
    long long smax = 1;          // accumulator slots of all levels (sum of S)

    bool adjoint = false;        // rings hold lambda; the FFT input is chi * lambda
    int adj_total = 0;           // segmented adjoint: forward steps N of the run
    int adj_done = 0;            //   adjoint steps done (tau)
    double* adj_gchi = nullptr;  //   dO/dchi accumulated so far (device, [M])

    // probe operator (probes.cu): element windows of every probe-voxel pair
    int n_probes = 0;
    double* probe_tab = nullptr;   // [P][6][WIN][M]
    int* probe_l0 = nullptr;       // [P][M]

    // PDSA operator A_n (pdsa.cu): kernel spectrum and diagonal of the last (n, flags)
    double* pdsa_spec = nullptr;   // [noct][6] unnormalised spectrum of sum_i c_i G_i
    double* pdsa_a = nullptr;      // [M] diagonal a_m (0 on voxels with chi = 0)
    double2* pdsa_xhat = nullptr;  // [3][nbins] spectrum scratch
    double* pdsa_conv = nullptr;   // [3][M] convolution scratch
    int pdsa_n = -1, pdsa_flags = -1;

    // counters and optional phase timing
    mot_stats stats = {};
    bool profiling = false;
    std::vector<cudaEvent_t> events;   // 6 per step of the current call

    cudaStream_t stream = nullptr;
    int device = 0;              // CUDA device the context was created on
    std::vector<mot_ctx*> rhs_ctx;   // further right-hand sides (mot_set_excitation_rhs):
                                     // contexts sharing this one's setup, owned by it
    mot_ctx* rhs_owner = nullptr;    // for such a right-hand side: the owning context
    int graph_steps = 0;         // steps per CUDA graph of the march (0: no graphs)
    cudaGraphExec_t gexec = nullptr;   // executable graph of one period, updated in place

    // mot_create_shared: setup (geometry, table, spectra, twiddles) borrowed from
    // shared_src, which must outlive this context; n_shared counts the borrowers
    mot_ctx* shared_src = nullptr;
    int n_shared = 0;
    int nsm = 0;
    int cg_blocks = 0;
    bool broken = false;
    std::string err;
};

template <typename R> inline HistoryBuffers<R>& hbuf(mot_ctx* c);
template <> inline HistoryBuffers<double>& hbuf<double>(mot_ctx* c) { return c->h64; }
template <> inline HistoryBuffers<float>& hbuf<float>(mot_ctx* c) { return c->h32; }

// ------------------------------------------------------------------ internals
namespace mot {

constexpr int WIN = 8;  // lag window per octant offset of the interaction table
constexpr int kPwTable = 1 << 16;   // nodes of the plane-wave table of one call
constexpr int kStatusWords = 8;     // device status words of a context (dstatus)
constexpr double kBarrierBudgetS = 2.0;   // longest wait at a grid barrier of the solve

// quadrature.cu
void compute_table(mot_ctx* c);
double* quad_windows(mot_ctx* c, const std::vector<int3>& tri);
void probe_windows(mot_ctx* c, int np, const int* probes, double* tab, int* l0);
// spectra.cu
void compute_spectra(mot_ctx* c);
void spectrum_of_lag(mot_ctx* c, int l, double* host_out);
void spectrum_of_combination(mot_ctx* c, const double* w_host, int n, bool round32,
                             double* dst);
// fft.cu
void fft_plan_axis(AxisFFT& a, int P);
void fft_free_axis(AxisFFT& a);
template <typename R>
void fft_forward(mot_ctx* c, const double* Jsoa, typename CT<R>::c* out, cudaStream_t s,
                 const double* scale = nullptr);
template <typename R>
void fft_inverse(mot_ctx* c, const typename CT<R>::c* in, R* out, cudaStream_t s);
// history.cu
// far levels of the blocked scheme for block B and ell (host only): level k covers
// lags [a[k], a[k] + S[k]); returns the number of levels, or -1 if more than 8 are needed
int level_plan(int block, int ell, bool fit, int S[8], int a[8]);
template <typename R> void history_alloc(mot_ctx* c);
template <typename R> void history_alloc_shared(mot_ctx* c, mot_ctx* src);
template <typename R> void history_free(mot_ctx* c);
// ev (optional, 3 events): recorded after the forward FFT, after the far-lag block
// products and after the near-lag MAC
template <typename R> void history_step(mot_ctx* c, int n, cudaStream_t s,
                                        cudaEvent_t* ev = nullptr);
template <typename R> void history_reset(mot_ctx* c, cudaStream_t s);
template <typename R> void level_spectra(mot_ctx* c);
// solve.cu
void solve_step(mot_ctx* c, int n, const double* En, double* norm2_out, cudaStream_t s);
void stencil_setup(mot_ctx* c);
void chebyshev_setup(mot_ctx* c);
void write_aos(mot_ctx* c, int n, double* out_dev, cudaStream_t s);
void read_aos(mot_ctx* c, const double* in_dev, double* slot, cudaStream_t s);
void history_out(mot_ctx* c, int n, double* out_dev, cudaStream_t s);
void adjoint_step(mot_ctx* c, int tau, int n, const double* g_aos, const double* J_aos,
                  int j_first, double* grad_chi, double* lam_out, double* norm2_out,
                  cudaStream_t s);
// excitation.cu
void excitation_setup(int dev);   // once per device: Gauss nodes of the voxel average
void plane_wave(mot_ctx* c, const double k[3], const double p[3], double fc, double st,
                double t0, int n_first, int n_steps, double* Edev, cudaStream_t s);

inline long long slot_index(long long n, long long R) { return ((n % R) + R) % R; }

}  // namespace mot

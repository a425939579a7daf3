// mot_plane_wave_static: the tested plane-wave excitation (Eq. E) delivered to host
// memory without allocating device memory.
//
// mot_plane_wave with a host destination evaluates the excitation into a device
// staging buffer that it cudaMalloc's and cudaFree's on every call.  Some callers must
// not allocate during a call: a process that reserves the device's memory up front
// for its own pool (a cudaMalloc could then fail part-way through a run), or a
// driver loop that cannot afford cudaFree's implicit device-wide synchronisation,
// which stalls every stream on the device.  This variant stages the result in one
// file-scope device array instead, so it allocates nothing, and it rejects requests
// larger than that array.
//
// The scratch array is resolved once per device (cudaGetSymbolAddress with that
// device current) on the first call there; that first call may also load the module,
// so make it before any stream capture on that device.  Each call runs on the device
// the context was created on (made current for the call, the caller's device restored
// afterwards), whichever device is current when it is made.  Nothing in the scratch needs
// to start at zero: the kernel writes every element that the copy then reads.  There
// is one scratch array per device per process, so calls that overlap in time (from
// several host threads, on any contexts of the same device) overwrite each other's
// staging data: serialise them.
#include <mutex>
#include <string>

#include "mot_internal.cuh"

namespace {

// 16 MiB of doubles: 3 M n_steps must not exceed this (e.g. 21 steps of a 32^3 grid)
constexpr long long kScratchDoubles = 2LL * 1024 * 1024;
__device__ __align__(256) double g_plane_wave_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// device address of the scratch array on device `dev` (resolved on first use)
cudaError_t scratch_on(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_plane_wave_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" mot_status mot_plane_wave_static(mot_ctx* c, const double k_hat[3],
                                            const double p_hat[3], double f_c, double sigma_t,
                                            double t0, int n_first, int n_steps, double* E_out,
                                            void* stream) {
    if (!c) return MOT_ERR_ARG;
    if (c->broken) return MOT_ERR_STATE;
    if (!k_hat || !p_hat || !E_out || n_steps < 1 || !(sigma_t > 0)) {
        c->err = "invalid plane-wave arguments";
        return MOT_ERR_ARG;
    }
    const long long need = 3LL * c->M * n_steps;
    if (need > kScratchDoubles) {
        c->err = "mot_plane_wave_static: 3 * M * n_steps = " + std::to_string(need) +
                 " doubles exceeds its fixed device scratch of " +
                 std::to_string(kScratchDoubles) + " doubles; request fewer steps per call";
        return MOT_ERR_ARG;
    }
    if (on_device(E_out)) {
        c->err = "mot_plane_wave_static writes host memory; use mot_plane_wave for a device "
                 "destination";
        return MOT_ERR_ARG;
    }
    // the context's device, made current for the call (and the caller's restored):
    // the scratch address and the launches must both belong to it
    if (c->device < 0 || c->device >= kMaxDevices) {
        c->err = "mot_plane_wave_static: context device beyond the supported range";
        return MOT_ERR_ARG;
    }
    int caller_dev = 0;
    cudaError_t e = cudaGetDevice(&caller_dev);
    if (e == cudaSuccess && caller_dev != c->device) e = cudaSetDevice(c->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("mot_plane_wave_static: cannot select the context's device: ") +
                 cudaGetErrorString(e);
        return MOT_ERR_CUDA;
    }
    struct Restore {
        int dev, prev;
        ~Restore() { if (dev != prev) cudaSetDevice(prev); }
    } restore{c->device, caller_dev};
    double* scratch = nullptr;
    e = scratch_on(c->device, &scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("mot_plane_wave_static: cudaGetSymbolAddress failed: ") +
                 cudaGetErrorString(e);
        return MOT_ERR_CUDA;
    }
    try {
        cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
        mot::plane_wave(c, k_hat, p_hat, f_c, sigma_t, t0, n_first, n_steps, scratch, s);
        MOT_CUDA_TRY(cudaMemcpyAsync(E_out, scratch, sizeof(double) * need,
                                     cudaMemcpyDeviceToHost, s));
        MOT_CUDA_TRY(cudaStreamSynchronize(s));
    } catch (const MotError& err) {
        c->err = err.msg;
        if (err.st == MOT_ERR_CUDA || err.st == MOT_ERR_TIMEOUT) c->broken = true;
        return err.st;
    }
    return MOT_OK;
}

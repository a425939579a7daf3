"""Python binding of the C ABI in include/mot.h (ctypes; argument marshalling only).

Every computation runs in the CUDA library libmot.so built in this directory by
``paper_2407_03323_gb300.build``.  If the library is missing the import of this
module's entry points raises: there is no CPU path.

Buffers may be numpy arrays (host memory) or torch CUDA tensors (device memory);
both are passed to the library as raw pointers.  Layouts follow the C ABI:
eps_r [W][V][U]; excitation and current densities [n][m][b] with
m = u + U (v + V w) and b = x, y, z.
"""
import ctypes
import os
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmot.so")

MOT_OK, MOT_ERR_ARG, MOT_ERR_OOM, MOT_ERR_CUDA = 0, 1, 2, 3
MOT_ERR_NOT_CONVERGED, MOT_ERR_UNSTABLE, MOT_ERR_TIMEOUT, MOT_ERR_STATE = 4, 5, 6, 7
STATUS_NAMES = {0: "MOT_OK", 1: "MOT_ERR_ARG", 2: "MOT_ERR_OOM", 3: "MOT_ERR_CUDA",
                4: "MOT_ERR_NOT_CONVERGED", 5: "MOT_ERR_UNSTABLE", 6: "MOT_ERR_TIMEOUT",
                7: "MOT_ERR_STATE"}
PRECISIONS = {"fp64": 0, "fp32_history": 1}
SCHEMES = {"direct": 0, "blocked": 1, "blocked_doubling": 2}

EXPORTS = ["mot_create", "mot_create_shared", "mot_destroy", "mot_set_excitation",
           "mot_plane_wave",
           "mot_plane_wave_static", "mot_march", "mot_restart", "mot_adjoint_begin",
           "mot_adjoint_run", "mot_adjoint_end",
           "mot_adjoint", "mot_eval_history", "mot_get_table", "mot_get_spectrum", "mot_get_info",
           "mot_get_levels", "mot_level_plan",
           "mot_set_solver", "mot_set_profiling", "mot_get_stats", "mot_pdsa_apply",
           "mot_pdsa_bounds", "mot_pdsa_lanczos", "mot_truncate_table", "mot_fir_magnitude",
           "mot_frequency_response", "mot_fma_peak", "mot_probe_setup", "mot_probe_field",
           "mot_probe_transpose", "mot_barrier_check", "mot_set_graph",
           "mot_set_excitation_rhs", "mot_march_rhs", "mot_rhs_context", "mot_create_padded",
           "mot_last_error"]
MOT_PDSA_FP32_SPECTRUM = 1
MOT_PDSA_FULL_REORTH = 2


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("mac_launches", ctypes.c_longlong),
                ("far_launches", ctypes.c_longlong), ("steps", ctypes.c_longlong),
                ("cg_iters", ctypes.c_longlong), ("ms_fft_fwd", ctypes.c_double),
                ("ms_far", ctypes.c_double), ("ms_mac", ctypes.c_double),
                ("ms_fft_inv", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("graph_launches", ctypes.c_longlong),
                ("graph_instantiations", ctypes.c_longlong)]


class MotError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


_lib = None


def load_library(path=LIB_PATH):
    """Load libmot.so and declare the signatures; raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmot.so not found at %s: run `python -m "
                           "paper_2407_03323_gb300.build` (there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    lib.mot_create.argtypes = [P, P, D, P, P, I, I, I, I, ctypes.POINTER(P)]
    lib.mot_destroy.argtypes = [P]
    lib.mot_destroy.restype = None
    lib.mot_set_excitation.argtypes = [P, I, P, P]
    lib.mot_plane_wave.argtypes = [P, P, P, D, D, D, I, I, P, P]
    lib.mot_plane_wave_static.argtypes = [P, P, P, D, D, D, I, I, P, P]
    lib.mot_march.argtypes = [P, I, P, P]
    lib.mot_eval_history.argtypes = [P, I, P, P, P]
    lib.mot_adjoint.argtypes = [P, I, P, P, P, P, P]
    lib.mot_adjoint_begin.argtypes = [P, I, P]
    lib.mot_adjoint_run.argtypes = [P, I, P, I, I, P, P, P]
    lib.mot_adjoint_end.argtypes = [P, P, P]
    lib.mot_restart.argtypes = [P, I, I, P, P]
    lib.mot_create_shared.argtypes = [P, ctypes.POINTER(P)]
    lib.mot_get_table.argtypes = [P, I, I, P]
    lib.mot_get_spectrum.argtypes = [P, I, P]
    lib.mot_get_info.argtypes = [P, P, P, P, P, P, P]
    lib.mot_get_levels.argtypes = [P, I, P, P, P]
    lib.mot_level_plan.argtypes = [I, I, I, I, P, P, P]
    lib.mot_set_solver.argtypes = [P, D, I, D]
    lib.mot_set_profiling.argtypes = [P, I]
    lib.mot_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.mot_pdsa_apply.argtypes = [P, I, I, P, P]
    lib.mot_pdsa_bounds.argtypes = [P, I, I, P]
    lib.mot_pdsa_lanczos.argtypes = [P, I, I, I, ctypes.c_ulonglong, I, P, P, P]
    lib.mot_truncate_table.argtypes = [P, D]
    lib.mot_fir_magnitude.argtypes = [P, I, I, P, P]
    lib.mot_frequency_response.argtypes = [I, I, P, D, D, P, D, D, I, P, P, P]
    lib.mot_fma_peak.argtypes = [I, I, P, P]
    lib.mot_probe_setup.argtypes = [P, I, P]
    lib.mot_probe_field.argtypes = [P, I, P, P, P]
    lib.mot_probe_transpose.argtypes = [P, I, P, P, P]
    lib.mot_barrier_check.argtypes = [I, I, I, D, P, P]
    lib.mot_set_graph.argtypes = [P, I]
    lib.mot_set_excitation_rhs.argtypes = [P, I, I, P, P]
    lib.mot_create_padded.argtypes = [P, P, D, P, P, I, I, I, I, P, P]
    lib.mot_march_rhs.argtypes = [P, I, P, P]
    lib.mot_rhs_context.argtypes = [P, I, P]
    lib.mot_last_error.argtypes = [P]
    lib.mot_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("mot_destroy", "mot_last_error"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _ptr(buf):
    """Raw pointer of a numpy array, a torch tensor, or an int; None -> NULL."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffers must be C-contiguous")
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        if hasattr(buf, "is_contiguous") and not buf.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return buf.data_ptr()
    raise TypeError("unsupported buffer type %r" % type(buf))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_ok(buf):
    if isinstance(buf, np.ndarray):
        return buf.dtype == np.float64
    dt = getattr(buf, "dtype", None)
    return dt is None or str(dt) == "torch.float64"


def fir_magnitude(taps, theta):
    """|sum_n exp(-i n theta) delta_n| (Eq. FIRmagnitude) at the normalised frequencies
    theta (mot_fir_magnitude)."""
    lib = load_library()
    t = np.ascontiguousarray(taps, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    out = np.zeros_like(th)
    st = lib.mot_fir_magnitude(t.ctypes.data if t.size else None, t.size, th.size,
                               th.ctypes.data, out.ctypes.data)
    if st != MOT_OK:
        raise MotError(st, "mot_fir_magnitude: invalid arguments")
    return out


def frequency_response(J, dt, taper, eps_probe, f_c, sigma_t, freqs, with_spectrum=False):
    """|H^alpha|(r, f) of Eq. Halpha from probe series J [N][n_probe][3] (numpy or CUDA
    tensor; mot_frequency_response): tapered over the last fraction `taper`, returns
    H [n_freq][n_probe][3] (and the complex j(f) with with_spectrum)."""
    lib = load_library()
    if isinstance(J, np.ndarray):
        J = np.ascontiguousarray(J, dtype=np.float64)
    n_steps, n_probe = J.shape[0], J.shape[1]
    e = np.ascontiguousarray(eps_probe, dtype=np.float64).reshape(-1)
    f = np.ascontiguousarray(freqs, dtype=np.float64).reshape(-1)
    H = np.zeros((f.size, n_probe, 3))
    jh = np.zeros((f.size, n_probe, 3), dtype=np.complex128) if with_spectrum else None
    st = lib.mot_frequency_response(n_steps, n_probe, _ptr(J), dt, taper, e.ctypes.data, f_c,
                                    sigma_t, f.size, f.ctypes.data, H.ctypes.data,
                                    None if jh is None else jh.ctypes.data)
    if st != MOT_OK:
        raise MotError(st, "mot_frequency_response failed")
    return (H, jh) if with_spectrum else H


def fma_peak(fp64=True, target_ms=100.0):
    """Sustained FMA rate of the current device in FLOP/s (mot_fma_peak), from one launch
    sized to take about target_ms after a short calibration launch."""
    lib = load_library()
    ms = ctypes.c_float()
    fl = ctypes.c_double()
    iters = 2048
    for _ in range(3):
        st = lib.mot_fma_peak(1 if fp64 else 0, iters, ctypes.byref(ms), ctypes.byref(fl))
        if st != MOT_OK:
            raise MotError(st, "mot_fma_peak failed")
        if ms.value >= 0.5 * target_ms:
            break
        iters = int(min(2 ** 30, iters * target_ms / max(ms.value, 1e-3)))
    return fl.value / (ms.value * 1e-3)


# FFT lengths with a compiled four-step codelet for the x, y and z passes
CODELET_LENGTHS = (64, 96, 210)


def smooth7(n):
    for r in (2, 3, 5, 7):
        while n % r == 0:
            n //= r
    return n == 1


def pad_size(N):
    """The library's default zero-padded FFT length for N voxels along an axis: the
    smallest even 7-smooth length >= 2 N - 1 (App. A)."""
    P = max(2 * N - 1, 2)
    while P % 2 or not smooth7(P):
        P += 1
    return P


def codelet_size(N, limit=1.5):
    """The smallest codelet length >= 2 N - 1 if it is at most `limit` times pad_size(N),
    else pad_size(N)."""
    p = pad_size(N)
    for c in CODELET_LENGTHS:
        if c >= 2 * N - 1 and c <= limit * p:
            return c
    return p


def level_plan(block, ell, scheme="blocked"):
    """The far levels [(S, first lag), ...] a context with this block size, ell and
    history scheme uses (mot_level_plan; host only, no device needed)."""
    lib = load_library()
    n = ctypes.c_int()
    S = (ctypes.c_int * 8)()
    a = (ctypes.c_int * 8)()
    st = lib.mot_level_plan(int(block), int(ell), SCHEMES[scheme], 8, ctypes.byref(n),
                            ctypes.cast(S, ctypes.c_void_p), ctypes.cast(a, ctypes.c_void_p))
    if st != MOT_OK:
        raise MotError(st, lib.mot_last_error(None).decode())
    return [(S[k], a[k]) for k in range(n.value)]


def barrier_check(n_blocks, rounds, absent=-1, budget_s=0.2):
    """One cooperative launch of the solve's grid barrier (mot_barrier_check): returns
    (status, blocks that passed every round, round of a timeout or 0)."""
    lib = load_library()
    passed = ctypes.c_int()
    rnd = ctypes.c_int()
    st = lib.mot_barrier_check(n_blocks, rounds, absent, budget_s, ctypes.byref(passed),
                               ctypes.byref(rnd))
    return st, passed.value, rnd.value


class Context:
    """A marching context (mot_create ... mot_destroy)."""

    def __init__(self, eps_r, taps=None, precision="fp64", scheme="direct", block=0, h=1.0,
                 fft_len=None):
        lib = load_library()
        eps = np.ascontiguousarray(np.asarray(eps_r, dtype=np.float64))
        if eps.ndim != 3:
            raise ValueError("eps_r must be [W][V][U]")
        W, V, U = eps.shape
        self.shape = (W, V, U)
        self.M = U * V * W
        grid = (ctypes.c_int * 3)(U, V, W)
        hh = (ctypes.c_double * 3)(h, h, h)
        t = np.ascontiguousarray(np.zeros(0) if taps is None else np.asarray(taps, np.float64))
        out = ctypes.c_void_p()
        fl = None if fft_len is None else (ctypes.c_int * 3)(*[int(v) for v in fft_len])
        st = lib.mot_create_padded(ctypes.cast(grid, ctypes.c_void_p),
                                   ctypes.cast(hh, ctypes.c_void_p), h, eps.ctypes.data,
                                   t.ctypes.data if t.size else None, int(t.size),
                                   PRECISIONS[precision], SCHEMES[scheme], int(block),
                                   None if fl is None else ctypes.cast(fl, ctypes.c_void_p),
                                   ctypes.byref(out))
        if st != MOT_OK:
            raise MotError(st, lib.mot_last_error(None).decode())
        self._h = out
        self._lib = lib
        self._scheme = scheme
        self._precision = precision
        self._block = int(block)
        info = self.info()
        self.ell = info["ell"]
        self.P = info["P"]

    # -- helpers
    def _check(self, st):
        if st != MOT_OK:
            raise MotError(st, self._lib.mot_last_error(self._h).decode())

    def share(self):
        """A second, independent marching state on this context's setup
        (mot_create_shared); this context is kept alive as long as the new one."""
        out = ctypes.c_void_p()
        st = self._lib.mot_create_shared(self._h, ctypes.byref(out))
        if st != MOT_OK:
            raise MotError(st, self._lib.mot_last_error(None).decode())
        c = Context.__new__(Context)
        c.shape, c.M, c._lib = self.shape, self.M, self._lib
        c._scheme, c._precision, c._block = self._scheme, self._precision, self._block
        c.ell, c.P = self.ell, self.P
        c._h = out
        c._src = self
        self._shares = [r for r in getattr(self, "_shares", []) if r() is not None]
        self._shares.append(weakref.ref(c))
        return c

    def close(self):
        """Destroy the context (mot_destroy); refused while contexts shared from it
        are alive.  A right-hand-side view (rhs) only drops its handle."""
        if getattr(self, "_borrowed", False):
            self._h = None
            return
        if getattr(self, "_h", None):
            live = [r() for r in getattr(self, "_shares", [])]
            if any(c is not None and getattr(c, "_h", None) for c in live):
                raise RuntimeError("close the contexts shared from this one first")
            self._lib.mot_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API
    def set_excitation(self, E, stream=None):
        """Stage E[n][M][3] (float64, numpy or CUDA tensor) for the next steps
        (mot_set_excitation); steps without staged excitation march with E = 0."""
        if not _dtype_ok(E):
            raise TypeError("E must be float64")
        n = E.shape[0]
        self._check_out(E, n)
        self._check(self._lib.mot_set_excitation(self._h, n, _ptr(E), _stream(stream)))

    def set_excitation_rhs(self, E, stream=None):
        """Stage E[r][n][M][3] (float64) for E.shape[0] right-hand sides
        (mot_set_excitation_rhs); right-hand side 0 is this context."""
        if not _dtype_ok(E):
            raise TypeError("E must be float64")
        n_rhs, n = E.shape[0], E.shape[1]
        self._check_out(E, n, n_rhs=n_rhs)
        self._check(self._lib.mot_set_excitation_rhs(self._h, n_rhs, n, _ptr(E), _stream(stream)))
        self._n_rhs = n_rhs

    def march_rhs(self, n_steps, out="host", stream=None):
        """March every right-hand side n_steps steps, interleaved (mot_march_rhs); out
        'host' returns J[r][n][M][3], None keeps J on the device, or pass a buffer."""
        n_rhs = getattr(self, "_n_rhs", 1)
        if isinstance(out, str):
            out = np.zeros((n_rhs, n_steps, self.M, 3))
        if out is not None:
            self._check_out(out, n_steps, n_rhs=n_rhs)
        self._check(self._lib.mot_march_rhs(self._h, n_steps, _ptr(out), _stream(stream)))
        return out

    def rhs(self, k):
        """The context of right-hand side k (mot_rhs_context), owned by this one: valid
        while this context is open."""
        out = ctypes.c_void_p()
        self._check(self._lib.mot_rhs_context(self._h, int(k), ctypes.byref(out)))
        if k == 0:
            return self
        c = Context.__new__(Context)
        c.shape, c.M, c._lib = self.shape, self.M, self._lib
        c._scheme, c._precision, c._block = self._scheme, self._precision, self._block
        c.ell, c.P = self.ell, self.P
        c._h = out
        c._borrowed = True
        c._owner = self
        return c

    def _check_out(self, out, n_steps, host_only=False, n_rhs=1):
        """The C side reads or writes n_rhs * n_steps * M * 3 doubles at `out`: refuse
        anything else."""
        is_np = isinstance(out, np.ndarray)
        if host_only and not (is_np or (hasattr(out, "device") and
                                        str(getattr(out, "device")) == "cpu")):
            raise TypeError("out must be host memory (a numpy array or a CPU tensor)")
        if not is_np and not hasattr(out, "data_ptr"):
            raise TypeError("out must be a numpy array or a torch tensor")
        if not _dtype_ok(out) or getattr(out, "dtype", None) is None:
            raise TypeError("out must be float64")
        size = out.size if is_np else out.numel()
        if size != n_rhs * n_steps * self.M * 3:
            raise ValueError("buffer holds %d values, %d needed ([%sn_steps][M][3])"
                             % (size, n_rhs * n_steps * self.M * 3, "n_rhs][" if n_rhs > 1 else ""))
        contiguous = out.flags["C_CONTIGUOUS"] if is_np else out.is_contiguous()
        if not contiguous:
            raise ValueError("out must be C-contiguous")

    def plane_wave(self, k_hat, p_hat, f_c, sigma_t, t0, n_first, n_steps, out=None, stream=None):
        """Tested modulated-Gaussian plane wave E[n_steps][M][3] of steps n_first..
        (mot_plane_wave, Eq. E); out: numpy array or CUDA tensor, else a new array."""
        if out is None:
            out = np.zeros((n_steps, self.M, 3))
        self._check_out(out, n_steps)
        k = np.ascontiguousarray(k_hat, dtype=np.float64)
        p = np.ascontiguousarray(p_hat, dtype=np.float64)
        self._check(self._lib.mot_plane_wave(self._h, k.ctypes.data, p.ctypes.data, f_c, sigma_t,
                                             t0, n_first, n_steps, _ptr(out), _stream(stream)))
        return out

    def plane_wave_static(self, k_hat, p_hat, f_c, sigma_t, t0, n_first, n_steps, out=None,
                          stream=None):
        """mot_plane_wave_static: as plane_wave, into host memory (numpy), staged in
        the library's fixed device scratch instead of a per-call allocation."""
        if out is None:
            out = np.zeros((n_steps, self.M, 3))
        self._check_out(out, n_steps, host_only=True)
        k = np.ascontiguousarray(k_hat, dtype=np.float64)
        p = np.ascontiguousarray(p_hat, dtype=np.float64)
        self._check(self._lib.mot_plane_wave_static(self._h, k.ctypes.data, p.ctypes.data, f_c,
                                                    sigma_t, t0, n_first, n_steps, _ptr(out),
                                                    _stream(stream)))
        return out

    def march(self, n_steps, out="host", stream=None):
        """March n_steps; out='host' returns a new numpy array, None keeps J on the
        device, or pass a preallocated numpy array / torch tensor."""
        if isinstance(out, str):
            out = np.zeros((n_steps, self.M, 3))
        if out is not None:
            self._check_out(out, n_steps)
        self._check(self._lib.mot_march(self._h, n_steps, _ptr(out), _stream(stream)))
        return out

    def adjoint(self, J, dO_dJ, want_lambda=False, stream=None):
        """dO/d eps_r per voxel by the adjoint march (mot_adjoint); returns grad [W][V][U]
        (and lambda [N][M][3] if want_lambda)."""
        if isinstance(J, np.ndarray):
            J = np.ascontiguousarray(J, dtype=np.float64)
        if isinstance(dO_dJ, np.ndarray):
            dO_dJ = np.ascontiguousarray(dO_dJ, dtype=np.float64)
        n = J.shape[0]
        grad = np.zeros(self.shape)
        lam = np.zeros((n, self.M, 3)) if want_lambda else None
        self._check(self._lib.mot_adjoint(self._h, n, _ptr(J), _ptr(dO_dJ), grad.ctypes.data,
                                          _ptr(lam), _stream(stream)))
        return (grad, lam) if want_lambda else grad

    def adjoint_begin(self, n_total, stream=None):
        """Open a segmented adjoint run of n_total forward steps (mot_adjoint_begin)."""
        self._check(self._lib.mot_adjoint_begin(self._h, n_total, _stream(stream)))

    def adjoint_run(self, n_count, J_win, win_first, dO_dJ, want_lambda=False, stream=None):
        """Advance the open adjoint run by n_count steps (mot_adjoint_run); J_win holds
        J_{win_first} .., dO_dJ the g_n of the n_count forward steps, oldest first."""
        if isinstance(J_win, np.ndarray):
            J_win = np.ascontiguousarray(J_win, dtype=np.float64)
        if isinstance(dO_dJ, np.ndarray):
            dO_dJ = np.ascontiguousarray(dO_dJ, dtype=np.float64)
        lam = np.zeros((n_count, self.M, 3)) if want_lambda else None
        self._check(self._lib.mot_adjoint_run(self._h, n_count, _ptr(J_win), win_first,
                                              J_win.shape[0], _ptr(dO_dJ), _ptr(lam),
                                              _stream(stream)))
        return lam

    def adjoint_end(self, want_grad=True, stream=None):
        """Close the adjoint run (mot_adjoint_end); returns dO/d eps_r [W][V][U]."""
        grad = np.zeros(self.shape) if want_grad else None
        self._check(self._lib.mot_adjoint_end(self._h, _ptr(grad), _stream(stream)))
        return grad

    def restart(self, n0, J_hist, stream=None):
        """Continue from a saved history (mot_restart): J_hist holds J_{n0-k+1} .. J_n0."""
        if isinstance(J_hist, np.ndarray):
            J_hist = np.ascontiguousarray(J_hist, dtype=np.float64)
        k = 0 if J_hist is None else J_hist.shape[0]
        self._check(self._lib.mot_restart(self._h, n0, k, _ptr(J_hist), _stream(stream)))

    def eval_history(self, J_hist, out=None, stream=None):
        """P_{n-1} = sum_l Z_l J_{n-l} for a given past J_hist[l-1] = J_{n-l}
        (mot_eval_history), through the same FFT / ring / MAC path as the march."""
        J = J_hist
        if isinstance(J, np.ndarray):
            J = np.ascontiguousarray(J, dtype=np.float64)
        if out is None:
            out = np.zeros((self.M, 3))
        self._check(self._lib.mot_eval_history(self._h, J.shape[0], _ptr(J), _ptr(out),
                                               _stream(stream)))
        return out

    def table(self, l0, n_lags):
        """Elements G_l^{ab}(d) of lags l0.. on the octant of offsets
        (mot_get_table): [n_lags][6][W][V][U], components xx yy zz xy xz yz."""
        W, V, U = self.shape
        out = np.zeros((n_lags, 6, W, V, U))
        self._check(self._lib.mot_get_table(self._h, l0, n_lags, out.ctypes.data))
        return out

    def spectrum(self, l):
        """Octant spectrum of lag l (mot_get_spectrum): [6][Pw/2+1][Pv/2+1][Pu/2+1],
        unnormalised."""
        Pu, Pv, Pw = self.P
        out = np.zeros((6, Pw // 2 + 1, Pv // 2 + 1, Pu // 2 + 1))
        self._check(self._lib.mot_get_spectrum(self._h, l, out.ctypes.data))
        return out

    def truncate_table(self, eps_trunc):
        """Round every element of the history lags l >= 1 to a multiple of eps_trunc
        (mot_truncate_table; before the first step)."""
        self._check(self._lib.mot_truncate_table(self._h, float(eps_trunc)))

    # ---------------------------------------------------------------- PDSA (Eq. Dn)
    def pdsa_apply(self, n, x, out=None, fp32_spectrum=False):
        """y = A_n x, A_n = diag(1/chi) D_n / C(ell, n) on the active voxels
        (mot_pdsa_apply); x, out [M][3] float64, numpy or CUDA tensor."""
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
        if out is None:
            out = np.zeros((self.M, 3))
        flags = MOT_PDSA_FP32_SPECTRUM if fp32_spectrum else 0
        self._check(self._lib.mot_pdsa_apply(self._h, n, flags, _ptr(x), _ptr(out)))
        return out

    def pdsa_bounds(self, n, fp32_spectrum=False):
        """Rigorous bracket of the spectrum of A_n from the circulant embedding
        (mot_pdsa_bounds)."""
        out = np.zeros(5)
        flags = MOT_PDSA_FP32_SPECTRUM if fp32_spectrum else 0
        self._check(self._lib.mot_pdsa_bounds(self._h, n, flags, out.ctypes.data))
        return {"lo": out[0], "hi": out[1], "symbol_min": out[2], "symbol_max": out[3],
                "chi_max": out[4]}

    def pdsa_lanczos(self, n, k, seed=0, fp32_spectrum=False, reorth=False, n_out=8):
        """k Lanczos steps on A_n (mot_pdsa_lanczos): the n_out smallest Ritz values
        (ascending), the extreme Ritz values with their residual norms, steps taken."""
        ritz = np.zeros(max(n_out, 1))
        info = (ctypes.c_int * 2)()
        ext = np.zeros(4)
        flags = (MOT_PDSA_FP32_SPECTRUM if fp32_spectrum else 0) | \
                (MOT_PDSA_FULL_REORTH if reorth else 0)
        self._check(self._lib.mot_pdsa_lanczos(self._h, n, flags, k, seed, n_out,
                                               ritz.ctypes.data,
                                               ctypes.cast(info, ctypes.c_void_p),
                                               ext.ctypes.data))
        return {"ritz": ritz[:info[0]].copy(), "theta_min": ext[0], "resid_min": ext[1],
                "theta_max": ext[2], "resid_max": ext[3], "steps": info[1]}

    # ---------------------------------------------------------------- probe field
    def probe_setup(self, probes):
        """Element windows of every probe-voxel pair (mot_probe_setup); probes are
        lattice indices (u, v, w), [n][3] ints, inside or outside the grid."""
        q = np.ascontiguousarray(np.asarray(probes, dtype=np.int32).reshape(-1, 3))
        self._check(self._lib.mot_probe_setup(self._h, q.shape[0], q.ctypes.data))
        self.n_probes = q.shape[0]

    def probe_field(self, J, out=None, stream=None):
        """Scattered field E[n][p][3] at the probes for currents J[n][M][3]
        (mot_probe_field); numpy arrays or CUDA tensors."""
        if isinstance(J, np.ndarray):
            J = np.ascontiguousarray(J, dtype=np.float64)
        if not _dtype_ok(J):
            raise TypeError("J must be float64")
        n = J.shape[0]
        if out is None:
            out = np.zeros((n, self.n_probes, 3))
        self._check(self._lib.mot_probe_field(self._h, n, _ptr(J), _ptr(out), _stream(stream)))
        return out

    def probe_transpose(self, W, out=None, stream=None):
        """Transposed probe operator g[k][M][3] applied to W[n][p][3]
        (mot_probe_transpose); numpy arrays or CUDA tensors."""
        if isinstance(W, np.ndarray):
            W = np.ascontiguousarray(W, dtype=np.float64)
        if not _dtype_ok(W):
            raise TypeError("W must be float64")
        n = W.shape[0]
        if out is None:
            out = np.zeros((n, self.M, 3))
        self._check(self._lib.mot_probe_transpose(self._h, n, _ptr(W), _ptr(out),
                                                  _stream(stream)))
        return out

    def _levels(self):
        n = ctypes.c_int()
        S = (ctypes.c_int * 8)()
        a = (ctypes.c_int * 8)()
        self._check(self._lib.mot_get_levels(self._h, 8, ctypes.byref(n),
                                             ctypes.cast(S, ctypes.c_void_p),
                                             ctypes.cast(a, ctypes.c_void_p)))
        return [(S[k], a[k]) for k in range(min(n.value, 8))]

    @property
    def levels(self):
        """Lengths S of the far levels of a blocked scheme (mot_get_levels; empty for
        the direct scheme)."""
        return [S for S, _ in self._levels()]

    @property
    def level_lags(self):
        """First lag of every far level (level k covers lags level_lags[k] ..
        level_lags[k] + levels[k] - 1)."""
        return [a for _, a in self._levels()]

    @property
    def period(self):
        """Steps after which the far levels' firing pattern repeats (the longest level;
        1 for the direct scheme)."""
        return max(self.levels, default=1)

    def info(self):
        """ell, padded sizes P, steps done, last ||J||, first failing step and the
        last CG iteration count (mot_get_info)."""
        ell = ctypes.c_int()
        P = (ctypes.c_int * 3)()
        nd = ctypes.c_int()
        ln = ctypes.c_double()
        fs = ctypes.c_int()
        it = ctypes.c_int()
        st = self._lib.mot_get_info(self._h, ctypes.byref(ell), ctypes.cast(P, ctypes.c_void_p),
                                    ctypes.byref(nd), ctypes.byref(ln), ctypes.byref(fs),
                                    ctypes.byref(it))
        self._check(st)
        return {"ell": ell.value, "P": tuple(P), "n_done": nd.value, "last_norm": ln.value,
                "fail_step": fs.value, "last_cg_iters": it.value}

    def set_graph(self, steps_per_graph):
        """March whole periods of steps_per_graph steps as CUDA graphs (mot_set_graph);
        0 turns graphs off.  For a blocked scheme a multiple of period."""
        self._check(self._lib.mot_set_graph(self._h, int(steps_per_graph)))

    def set_profiling(self, enable=True):
        """Per-phase event timing in march and counter reset (mot_set_profiling)."""
        self._check(self._lib.mot_set_profiling(self._h, 1 if enable else 0))

    def stats(self):
        """Launch, step and CG counters and the per-phase times (mot_get_stats)."""
        st = Stats()
        self._check(self._lib.mot_get_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def set_solver(self, tol=None, max_iter=200, growth_limit=1e12):
        """Z_0 solve tolerance (default 1e-13 FP64, 3e-8 FP32-history), inner
        iteration cap and the growth limit of the stability monitor (mot_set_solver)."""
        if tol is None:
            tol = 1e-13 if self._precision == "fp64" else 3e-8
        self._check(self._lib.mot_set_solver(self._h, tol, max_iter, growth_limit))

"""ctypes binding of libbl.so with the C function names of include/bl.h.

Argument marshalling only: every step of the tracking path runs in the CUDA
library. Device memory and streams come from torch.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbl.so")

BL_OK, BL_ERR_INVALID_ARG, BL_ERR_CUDA, BL_ERR_OOM = 0, 1, 2, 3
BL_ERR_UNSUPPORTED_ARCH, BL_ERR_NONFINITE, BL_ERR_TIMEOUT, BL_ERR_STATE = 4, 5, 6, 7
BL_F32, BL_F64 = 0, 1
BL_DRIFT, BL_QUAD, BL_SBEND, BL_PLASMA, BL_PLASMA_LENS = 0, 1, 2, 3, 4
BL_OBJ_EPS_N_X, BL_OBJ_SIGMA_X, BL_OBJ_EPS_N_Y, BL_OBJ_SIGMA_Y = 0, 1, 2, 3
BL_MLP_NPARAM = 51206
OBJECTIVES = {"eps_n_x": 0, "sigma_x": 1, "eps_n_y": 2, "sigma_y": 3}
KINDS = {"drift": BL_DRIFT, "quad": BL_QUAD, "sbend": BL_SBEND, "plasma": BL_PLASMA,
         "plasma_lens": BL_PLASMA_LENS}
WIDTHS = (6, 128, 128, 128, 128, 6)


class BlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libbl status %d: %s" % (status, msg))
        self.status = status


class bl_bunch(C.Structure):
    _fields_ = [("x", C.c_void_p), ("px", C.c_void_p), ("y", C.c_void_p), ("py", C.c_void_p),
                ("t", C.c_void_p), ("pt", C.c_void_p), ("n", C.c_int64), ("n_bunch", C.c_int32),
                ("dtype", C.c_int32), ("offsets_dev", C.c_void_p), ("offsets_host", C.c_void_p),
                ("gamma_ref", C.c_double)]


class bl_element(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nsteps", C.c_int32), ("L", C.c_double), ("k", C.c_double),
                ("angle", C.c_double), ("n0_cm3", C.c_double), ("E0_Vpm", C.c_double),
                ("phi0", C.c_double), ("surrogate", C.c_void_p), ("per_bunch_k", C.c_void_p),
                ("wide_surrogate", C.c_void_p)]


class bl_mlp_desc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("widths", C.POINTER(C.c_int32)),
                ("W", C.POINTER(C.POINTER(C.c_float))), ("b", C.POINTER(C.POINTER(C.c_float))),
                ("mu_in", C.POINTER(C.c_double)), ("sd_in", C.POINTER(C.c_double)),
                ("mu_out", C.POINTER(C.c_double)), ("sd_out", C.POINTER(C.c_double))]


class bl_wide_mlp_desc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("widths", C.POINTER(C.c_int32)),
                ("W", C.POINTER(C.POINTER(C.c_float))), ("b", C.POINTER(C.POINTER(C.c_float))),
                ("slopes", C.POINTER(C.c_float)),
                ("mu_in", C.POINTER(C.c_double)), ("sd_in", C.POINTER(C.c_double)),
                ("mu_out", C.POINTER(C.c_double)), ("sd_out", C.POINTER(C.c_double))]


class bl_adam_cfg(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double)]


_lib = None
_P, _I64, _I32, _D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
_SIGS = {
    "bl_lattice_create": ([_P, _I32, _I32, _P], C.c_int),
    "bl_lattice_destroy": ([_P], C.c_int),
    "bl_lattice_num_elements": ([_P], C.c_int32),
    "bl_lattice_num_quads": ([_P], C.c_int32),
    "bl_track": ([_P, _P, _P, _P, _P], C.c_int),
    "bl_moments": ([_P, _P, _P], C.c_int),
    "bl_moments_noalloc": ([_P, _P, _P], C.c_int),
    "bl_apply_linear": ([_P, _P, _I32, _P], C.c_int),
    "bl_push_stage": ([_P, _P, _P], C.c_int),
    "bl_reference_exit": ([_P, _D, _P], C.c_int),
    "bl_segment_matrix": ([_P, _I32, _D, _P], C.c_int),
    "bl_beam_quantities": ([_P, _D, _P], C.c_int),
    "bl_surrogate_create": ([_P, _P], C.c_int),
    "bl_surrogate_destroy": ([_P], C.c_int),
    "bl_surrogate_set_domain": ([_P, _P, _P], C.c_int),
    "bl_surrogate_save": ([_P, C.c_char_p], C.c_int),
    "bl_surrogate_load": ([C.c_char_p, _P], C.c_int),
    "bl_surrogate_get_norm": ([_P, _P, _P, _P, _P], C.c_int),
    "bl_surrogate_get_domain": ([_P, _P, _P, _P], C.c_int),
    "bl_surrogate_get_params": ([_P, _P, _P], C.c_int),
    "bl_surrogate_apply": ([_P, _P, _P], C.c_int),
    "bl_surrogate_train_step": ([_P, _P, _P, _I64, _P, _I64, _P, _P, _P], C.c_int),
    "bl_surrogate_grad": ([_P, _P, _P, _I64, _P, _I64, _P, _P, _P], C.c_int),
    "bl_surrogate_loss": ([_P, _P, _P, _I64, _P, _I64, _P, _P], C.c_int),
    "bl_track_grad": ([_P, _P, _I32, _P, _P, _P], C.c_int),
    "bl_track_num_reductions": ([_P], C.c_int32),
    "bl_track_async": ([_P, _P, _P, _P], C.c_int),
    "bl_track_host": ([_P, _P, C.c_int64, _P, _P, C.c_int64, _P, _P, _P], C.c_int),
    "bl_track_expand_moments": ([_P, _I32, _P, _P], C.c_int),
    "bl_wide_mlp_create": ([_P, _P], C.c_int),
    "bl_wide_mlp_destroy": ([_P], C.c_int),
    "bl_wide_mlp_apply": ([_P, _P, _I64, _P], C.c_int),
    "bl_wide_mlp_num_params": ([_P, _P], C.c_int),
    "bl_wide_mlp_grad": ([_P, _P, _P, _I64, _P, _I64, _P, _P, _P], C.c_int),
    "bl_wide_mlp_train_step": ([_P, _P, _P, _I64, _P, _I64, _P, _P, _P], C.c_int),
    "bl_wide_mlp_get_params": ([_P, _P, _P, _P], C.c_int),
    "bl_last_error_message": ([], C.c_char_p),
    "bl_version": ([], C.c_char_p),
    "bl_poll_device_errors": ([], C.c_int),
    "bl_debug_fail_allocations": ([C.c_int], C.c_int),
    "bl_debug_train_kernel": ([C.c_int], C.c_int),
    "bl_debug_pool_moments": ([_P, C.c_int32, _P], C.c_int),
}


def lib():
    """Load libbl.so (built by paper_2402_17248_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libbl.so is not built (%s); run paper_2402_17248_gb300.build"
                               % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(st):
    if st != BL_OK:
        raise BlError(st, lib().bl_last_error_message().decode())
    return st


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ bunches
class Bunch:
    """Six device tensors of one dtype plus the host reference gamma (bl_bunch)."""

    def __init__(self, coords, gamma_ref, offsets=None):
        import torch
        assert len(coords) == 6
        self.coords = list(coords)
        dt = coords[0].dtype
        assert all(c.dtype == dt and c.is_cuda and c.is_contiguous() and c.numel() == coords[0].numel()
                   for c in coords)
        self.struct = bl_bunch()
        for name, c in zip(("x", "px", "y", "py", "t", "pt"), coords):
            setattr(self.struct, name, c.data_ptr())
        self.struct.n = coords[0].numel()
        self.struct.dtype = BL_F32 if dt == torch.float32 else BL_F64
        self.struct.gamma_ref = float(gamma_ref)
        if offsets is None:
            self.struct.n_bunch = 1
            self.offsets_host = None
            self.offsets_dev = None
        else:
            self.offsets_host = np.ascontiguousarray(offsets, dtype=np.int64)
            self.offsets_dev = torch.tensor(self.offsets_host, device=coords[0].device)
            self.struct.n_bunch = len(self.offsets_host) - 1
            self.struct.offsets_dev = self.offsets_dev.data_ptr()
            self.struct.offsets_host = self.offsets_host.ctypes.data

    @property
    def gamma_ref(self):
        return self.struct.gamma_ref

    @property
    def n_bunch(self):
        return self.struct.n_bunch

    def ref(self):
        return C.byref(self.struct)


# ----------------------------------------------------------------- lattices
def make_elements(elements):
    """Element dicts (kind, L, k, angle, nsteps, n0_cm3, E0_Vpm, phi0,
    surrogate, per_bunch_k) -> ctypes array plus owned buffers."""
    arr = (bl_element * len(elements))()
    keep = []
    for i, e in enumerate(elements):
        s = arr[i]
        s.kind = KINDS[e["kind"]]
        s.L = e.get("L", 0.0)
        s.k = e.get("k", 0.0)
        s.angle = e.get("angle", 0.0)
        s.nsteps = e.get("nsteps", 0)
        s.n0_cm3 = e.get("n0_cm3", 0.0)
        s.E0_Vpm = e.get("E0_Vpm", 0.0)
        s.phi0 = e.get("phi0", 0.0)
        sur = e.get("surrogate")
        if isinstance(sur, WideSurrogate):
            s.wide_surrogate = sur.handle.value
        else:
            s.surrogate = sur.handle.value if sur is not None else None
        pbk = e.get("per_bunch_k")
        if pbk is not None:
            a = np.ascontiguousarray(pbk, dtype=np.float64)
            keep.append(a)
            s.per_bunch_k = a.ctypes.data
    return arr, keep


class Lattice:
    def __init__(self, elements, n_bunch_k=0):
        self.elements = elements
        arr, keep = make_elements(elements)
        self.handle = C.c_void_p()
        _check(lib().bl_lattice_create(arr, len(elements), n_bunch_k, C.byref(self.handle)))
        self._surrogates = [e.get("surrogate") for e in elements]

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bl_lattice_destroy(self.handle)
            self.handle = None

    @property
    def num_elements(self):
        return lib().bl_lattice_num_elements(self.handle)

    @property
    def num_quads(self):
        return lib().bl_lattice_num_quads(self.handle)


def bl_lattice_create(elements, n_bunch_k=0):
    return Lattice(elements, n_bunch_k)


def bl_track(bunch, lattice, moments=True, stream=None):
    """Returns (moments [n_el][n_bunch][28] or None, nonfinite count or None)."""
    m = None
    nf = C.c_int64(0)
    if moments:
        m = np.zeros((lattice.num_elements, bunch.n_bunch, 28))
    st = lib().bl_track(bunch.ref(), lattice.handle, m.ctypes.data if m is not None else None,
                        C.byref(nf) if moments else None, _stream(stream))
    if st not in (BL_OK, BL_ERR_NONFINITE):
        _check(st)
    return m, (nf.value if moments else None)


def _host_ptr(a):
    """Address of a host float32 buffer: a CPU torch tensor or a numpy array."""
    if hasattr(a, "data_ptr"):
        if a.is_cuda or a.dtype.itemsize != 4 or not a.is_contiguous():
            raise ValueError("host coordinates must be contiguous CPU float32 tensors")
        return a.data_ptr()
    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host coordinates must be contiguous float32 arrays")
    return a.ctypes.data


def bl_track_host(coords_in, coords_out, gamma_ref, lattice, chunk=0, moments=True, stream=None):
    """Track a host-resident FP32 bunch (6 arrays or CPU tensors, page-locked
    for overlap; coords_out may be coords_in) through the lattice in chunks
    streamed through the GPU. Returns (moments [n_el][1][28] or None,
    nonfinite count or None, gamma_ref at the exit)."""
    if len(coords_in) != 6 or len(coords_out) != 6:
        raise ValueError("need 6 input and 6 output coordinate arrays")
    n = len(coords_in[0])
    if any(len(a) != n for a in list(coords_in) + list(coords_out)):
        raise ValueError("coordinate arrays differ in length")
    pin = (C.c_void_p * 6)(*[_host_ptr(a) for a in coords_in])
    pout = (C.c_void_p * 6)(*[_host_ptr(a) for a in coords_out])
    g = C.c_double(gamma_ref)
    nf = C.c_int64(0)
    m = np.zeros((lattice.num_elements, 1, 28)) if moments else None
    st = lib().bl_track_host(pin, pout, n, C.byref(g), lattice.handle, int(chunk),
                             m.ctypes.data if m is not None else None,
                             C.byref(nf) if moments else None, _stream(stream))
    if st not in (BL_OK, BL_ERR_NONFINITE):
        _check(st)
    return m, (nf.value if moments else None), g.value


def bl_track_async(bunch, lattice, reduced=None, stream=None):
    """Enqueue bl_track without synchronising (capturable in a CUDA graph);
    reduced: device float64 tensor of reduced_size(lattice, bunch) or None."""
    _check(lib().bl_track_async(bunch.ref(), lattice.handle,
                                _ptr(reduced) if reduced is not None else None, _stream(stream)))


def reduced_size(lattice, bunch):
    return lib().bl_track_num_reductions(lattice.handle) * bunch.n_bunch * 28 + 1


def bl_track_expand_moments(lattice, n_bunch, reduced_host):
    """Moments [n_el][n_bunch][28] and the non-finite count from the raw
    reductions copied back from bl_track_async."""
    r = np.ascontiguousarray(reduced_host, dtype=np.float64)
    m = np.zeros((lattice.num_elements, n_bunch, 28))
    _check(lib().bl_track_expand_moments(lattice.handle, n_bunch, r.ctypes.data, m.ctypes.data))
    return m, int(r[-1:].view(np.uint64)[0])


class TrackGraph:
    """bl_track of one bunch through one lattice captured as a CUDA graph:
    replay() re-runs every launch of the pass (the bunch must hold new input
    particles at the captured entry energy); moments() returns the moments of
    the last replay."""

    def __init__(self, bunch, lattice):
        import torch
        self.bunch, self.lattice = bunch, lattice
        self.gamma_in = bunch.gamma_ref
        self.reduced = torch.zeros(reduced_size(lattice, bunch), dtype=torch.float64,
                                   device=bunch.coords[0].device)
        # the library's work buffers belong to a stream: warm up on the
        # stream that is then captured
        self.stream = torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            bl_track_async(bunch, lattice, self.reduced)   # plan and work buffers
        torch.cuda.synchronize()
        bunch.struct.gamma_ref = self.gamma_in
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            bl_track_async(bunch, lattice, self.reduced)
        self.gamma_out = bunch.gamma_ref

    def replay(self):
        self.graph.replay()
        self.bunch.struct.gamma_ref = self.gamma_out

    def moments(self):
        import torch
        torch.cuda.synchronize()
        return bl_track_expand_moments(self.lattice, self.bunch.n_bunch,
                                       self.reduced.cpu().numpy())


def bl_moments(bunch, out=None, stream=None):
    """Moments [n_bunch][28] into a host array (synchronises the stream)."""
    import torch
    h = np.zeros((bunch.n_bunch, 28)) if out is None else out
    _check(lib().bl_moments(bunch.ref(), h.ctypes.data, _stream(stream)))
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return h


def bl_moments_noalloc(bunch, out, stream=None):
    """Moments into `out` (a contiguous CUDA float64 tensor of at least
    n_bunch*28 elements) using the library's fixed scratch array instead of
    any allocation."""
    import torch
    if not isinstance(out, torch.Tensor) or not out.is_cuda:
        raise BlError(BL_ERR_INVALID_ARG, "out must be a CUDA tensor")
    if out.dtype != torch.float64 or not out.is_contiguous():
        raise BlError(BL_ERR_INVALID_ARG, "out must be a contiguous float64 tensor")
    if out.numel() < bunch.n_bunch * 28:
        raise BlError(BL_ERR_INVALID_ARG, "out holds %d doubles, %d needed"
                      % (out.numel(), bunch.n_bunch * 28))
    _check(lib().bl_moments_noalloc(bunch.ref(), _ptr(out), _stream(stream)))


def bl_apply_linear(bunch, M, stream=None):
    M = np.ascontiguousarray(M, dtype=np.float64)
    per = 1 if M.ndim == 3 else 0
    _check(lib().bl_apply_linear(bunch.ref(), M.ctypes.data, per, _stream(stream)))


def bl_push_stage(bunch, stage, stream=None):
    arr, keep = make_elements([stage])
    _check(lib().bl_push_stage(bunch.ref(), arr, _stream(stream)))
    return bunch.gamma_ref


def bl_reference_exit(stage, gamma_in):
    arr, keep = make_elements([stage])
    g = C.c_double()
    _check(lib().bl_reference_exit(arr, float(gamma_in), C.byref(g)))
    return g.value


def bl_segment_matrix(elements, gamma_ref):
    """FP64 6x6 transfer matrix of a run of linear elements (host)."""
    arr, keep = make_elements(elements) if elements else (None, [])
    M = np.zeros((6, 6))
    _check(lib().bl_segment_matrix(arr, len(elements), float(gamma_ref), M.ctypes.data))
    return M


BEAM_QUANTITIES = ("eps_n_x", "eps_n_y", "sigma_x", "sigma_y", "mean_gamma", "rel_energy_spread")


def bl_beam_quantities(m28, gamma_ref):
    m = np.ascontiguousarray(m28, dtype=np.float64)
    out = np.zeros(6)
    _check(lib().bl_beam_quantities(m.ctypes.data, float(gamma_ref), out.ctypes.data))
    return dict(zip(BEAM_QUANTITIES, out.tolist()))


# --------------------------------------------------------------- surrogates
class Surrogate:
    """bl_surrogate handle built from weights W[l] (out x in), biases b[l] and
    FP64 normalisation constants."""

    def __init__(self, Ws, bs, mu_in, sd_in, mu_out, sd_out):
        Wf = [np.ascontiguousarray(W, dtype=np.float32) for W in Ws]
        bf = [np.ascontiguousarray(b, dtype=np.float32) for b in bs]
        nrm = [np.ascontiguousarray(v, dtype=np.float64) for v in (mu_in, sd_in, mu_out, sd_out)]
        widths = (C.c_int32 * 6)(*WIDTHS)
        Wp = (C.POINTER(C.c_float) * 5)(*[w.ctypes.data_as(C.POINTER(C.c_float)) for w in Wf])
        bp = (C.POINTER(C.c_float) * 5)(*[b.ctypes.data_as(C.POINTER(C.c_float)) for b in bf])
        d = bl_mlp_desc()
        d.n_layers = 5
        d.widths = widths
        d.W = Wp
        d.b = bp
        d.mu_in, d.sd_in, d.mu_out, d.sd_out = [v.ctypes.data_as(C.POINTER(C.c_double)) for v in nrm]
        self.handle = C.c_void_p()
        _check(lib().bl_surrogate_create(C.byref(d), C.byref(self.handle)))
        self.mu_in, self.sd_in, self.mu_out, self.sd_out = nrm
        self.domain = None

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bl_surrogate_destroy(self.handle)
            self.handle = None

    def save(self, path):
        """Write a surrogate file (parameters, Adam state, normalisation, domain)."""
        _check(lib().bl_surrogate_save(self.handle, os.fsencode(path)))

    @classmethod
    def load(cls, path):
        """A surrogate from a file written by save(); training can resume."""
        self = cls.__new__(cls)
        self.handle = C.c_void_p()
        _check(lib().bl_surrogate_load(os.fsencode(path), C.byref(self.handle)))
        nrm = [np.zeros(6) for _ in range(4)]
        _check(lib().bl_surrogate_get_norm(self.handle, *[v.ctypes.data for v in nrm]))
        self.mu_in, self.sd_in, self.mu_out, self.sd_out = nrm
        lo, hi, has = np.zeros(6), np.zeros(6), C.c_int32(0)
        _check(lib().bl_surrogate_get_domain(self.handle, lo.ctypes.data, hi.ctypes.data,
                                             C.byref(has)))
        self.domain = (lo, hi) if has.value else None
        return self

    def set_domain(self, lo, hi):
        """Training-input box (raw coordinates); None clears it."""
        if lo is None:
            _check(lib().bl_surrogate_set_domain(self.handle, None, None))
            self.domain = None
            return
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        _check(lib().bl_surrogate_set_domain(self.handle, lo.ctypes.data, hi.ctypes.data))
        self.domain = (lo, hi)

    def params(self):
        Ws = [np.zeros((WIDTHS[l + 1], WIDTHS[l]), dtype=np.float32) for l in range(5)]
        bs = [np.zeros(WIDTHS[l + 1], dtype=np.float32) for l in range(5)]
        Wp = (C.POINTER(C.c_float) * 5)(*[w.ctypes.data_as(C.POINTER(C.c_float)) for w in Ws])
        bp = (C.POINTER(C.c_float) * 5)(*[b.ctypes.data_as(C.POINTER(C.c_float)) for b in bs])
        _check(lib().bl_surrogate_get_params(self.handle, Wp, bp))
        return Ws, bs


class WideSurrogate:
    """bl_wide_mlp handle: the paper's PReLU networks of any widths
    6 -> H ... H -> 6 (weights W[l] out x in, biases b[l], one slope per
    hidden layer, FP64 normalisation constants)."""

    def __init__(self, Ws, bs, slopes, mu_in, sd_in, mu_out, sd_out):
        L = len(Ws)
        Wf = [np.ascontiguousarray(W, dtype=np.float32) for W in Ws]
        bf = [np.ascontiguousarray(b, dtype=np.float32) for b in bs]
        sl = np.ascontiguousarray(slopes, dtype=np.float32)
        nrm = [np.ascontiguousarray(v, dtype=np.float64) for v in (mu_in, sd_in, mu_out, sd_out)]
        self.widths = [Wf[0].shape[1]] + [W.shape[0] for W in Wf]
        widths = (C.c_int32 * (L + 1))(*self.widths)
        Wp = (C.POINTER(C.c_float) * L)(*[w.ctypes.data_as(C.POINTER(C.c_float)) for w in Wf])
        bp = (C.POINTER(C.c_float) * L)(*[b.ctypes.data_as(C.POINTER(C.c_float)) for b in bf])
        d = bl_wide_mlp_desc()
        d.n_layers = L
        d.widths = widths
        d.W = Wp
        d.b = bp
        d.slopes = sl.ctypes.data_as(C.POINTER(C.c_float))
        d.mu_in, d.sd_in, d.mu_out, d.sd_out = [v.ctypes.data_as(C.POINTER(C.c_double)) for v in nrm]
        self.handle = C.c_void_p()
        _check(lib().bl_wide_mlp_create(C.byref(d), C.byref(self.handle)))
        self.mu_in, self.sd_in, self.mu_out, self.sd_out = [np.array(v) for v in nrm]
        self.domain = None

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bl_wide_mlp_destroy(self.handle)
            self.handle = None

    @property
    def num_params(self):
        n = C.c_int64(0)
        _check(lib().bl_wide_mlp_num_params(self.handle, C.byref(n)))
        return n.value

    def params(self):
        """(weights [out x in], biases, slopes) of the FP32 masters."""
        L = len(self.widths) - 1
        Ws = [np.zeros((self.widths[l + 1], self.widths[l]), dtype=np.float32) for l in range(L)]
        bs = [np.zeros(self.widths[l + 1], dtype=np.float32) for l in range(L)]
        sl = np.zeros(L - 1, dtype=np.float32)
        Wp = (C.POINTER(C.c_float) * L)(*[w.ctypes.data_as(C.POINTER(C.c_float)) for w in Ws])
        bp = (C.POINTER(C.c_float) * L)(*[b.ctypes.data_as(C.POINTER(C.c_float)) for b in bs])
        _check(lib().bl_wide_mlp_get_params(self.handle, Wp, bp, sl.ctypes.data))
        return Ws, bs, sl


def bl_wide_mlp_apply(net, bunch, chunk=0, stream=None):
    _check(lib().bl_wide_mlp_apply(net.handle, bunch.ref(), int(chunk), _stream(stream)))


def bl_wide_mlp_grad(net, inp, out, grad_out, idx=None, batch=None, loss_out=None, stream=None):
    """inp, out: device float32 [6, ld]; grad_out: device float32 [num_params]."""
    ld = inp.shape[1]
    if batch is None:
        batch = idx.numel() if idx is not None else ld
    _check(lib().bl_wide_mlp_grad(net.handle, _ptr(inp), _ptr(out), ld, _ptr(idx), batch,
                                  _ptr(grad_out), _ptr(loss_out), _stream(stream)))


def bl_wide_mlp_train_step(net, inp, out, idx=None, batch=None, lr=1e-4, beta1=0.9,
                           beta2=0.999, eps=1e-8, loss_out=None, stream=None):
    assert inp.is_contiguous() and out.is_contiguous() and inp.shape == out.shape
    ld = inp.shape[1]
    if batch is None:
        batch = idx.numel() if idx is not None else ld
    cfg = bl_adam_cfg(lr, beta1, beta2, eps)
    _check(lib().bl_wide_mlp_train_step(net.handle, _ptr(inp), _ptr(out), ld, _ptr(idx), batch,
                                        C.byref(cfg), _ptr(loss_out), _stream(stream)))


def bl_surrogate_create(Ws, bs, mu_in, sd_in, mu_out, sd_out):
    return Surrogate(Ws, bs, mu_in, sd_in, mu_out, sd_out)


def bl_surrogate_apply(sur, bunch, stream=None):
    _check(lib().bl_surrogate_apply(sur.handle, bunch.ref(), _stream(stream)))


def bl_surrogate_train_step(sur, inp, out, idx=None, batch=None, lr=1e-4, beta1=0.9,
                            beta2=0.999, eps=1e-8, loss_out=None, stream=None):
    """inp, out: device float32 [6, ld]; idx: device int64 [batch] or None."""
    assert inp.is_contiguous() and out.is_contiguous() and inp.shape == out.shape
    ld = inp.shape[1]
    if batch is None:
        batch = idx.numel() if idx is not None else ld
    cfg = bl_adam_cfg(lr, beta1, beta2, eps)
    _check(lib().bl_surrogate_train_step(sur.handle, _ptr(inp), _ptr(out), ld, _ptr(idx), batch,
                                         C.byref(cfg), _ptr(loss_out), _stream(stream)))


def bl_surrogate_grad(sur, inp, out, grad_out, idx=None, batch=None, loss_out=None, stream=None):
    ld = inp.shape[1]
    if batch is None:
        batch = idx.numel() if idx is not None else ld
    _check(lib().bl_surrogate_grad(sur.handle, _ptr(inp), _ptr(out), ld, _ptr(idx), batch,
                                   _ptr(grad_out), _ptr(loss_out), _stream(stream)))


def bl_surrogate_loss(sur, inp, out, loss_out, idx=None, count=None, stream=None):
    ld = inp.shape[1]
    if count is None:
        count = idx.numel() if idx is not None else ld
    _check(lib().bl_surrogate_loss(sur.handle, _ptr(inp), _ptr(out), ld, _ptr(idx), count,
                                   _ptr(loss_out), _stream(stream)))


def bl_track_grad(bunch, lattice, objective="eps_n_x", stream=None):
    """Returns (J [n_bunch], dJ/dk [n_bunch][n_quads])."""
    J = np.zeros(bunch.n_bunch)
    g = np.zeros((bunch.n_bunch, lattice.num_quads))
    _check(lib().bl_track_grad(bunch.ref(), lattice.handle, OBJECTIVES[objective], J.ctypes.data,
                               g.ctypes.data, _stream(stream)))
    return J, g


def bl_poll_device_errors():
    _check(lib().bl_poll_device_errors())


def bl_version():
    return lib().bl_version().decode()


def bl_debug_fail_allocations(n):
    return lib().bl_debug_fail_allocations(int(n))


def bl_debug_train_kernel(simt):
    """Select the SIMT FP32 (True) or tensor-core (False, default) gradient
    kernel behind bl_surrogate_train_step / bl_surrogate_grad; returns the
    previous setting."""
    return bool(lib().bl_debug_train_kernel(1 if simt else 0))


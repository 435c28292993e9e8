"""Python binding of the fasttracks C ABI (include/fasttracks.h) for B300 / sm_103a.

Argument marshalling only: every step of the search runs in libfasttracks.so's CUDA
kernels.  Function names follow the C ABI without the ``ft_`` prefix.  Arrays may be numpy
arrays (host memory) or torch tensors (device tensors on the context's device are passed
as device pointers; the call is then asynchronous on ``stream``, by default torch's current
stream).  If the library is not built the import still works but every call raises
FtError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("FASTTRACKS_LIB") or os.path.join(_HERE, "libfasttracks.so")

FT_F32, FT_F16, FT_BF16, FT_F64 = 0, 1, 2, 3
DTYPES = {"f32": FT_F32, "f16": FT_F16, "bf16": FT_BF16}
ERRORS = {-1: "FT_ERR_ARG", -2: "FT_ERR_CUDA", -3: "FT_ERR_OOM", -4: "FT_ERR_TIMEOUT",
          -5: "FT_ERR_RANGE", -6: "FT_ERR_UNSUPPORTED"}

# ft_candidate {int64 template_idx; float s; float z}
CANDIDATE_DTYPE = np.dtype([("template_idx", "<i8"), ("s", "<f4"), ("z", "<f4")])


class FtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _BandDesc(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int), ("n_sft", ctypes.POINTER(ctypes.c_int)),
                ("n_bins", ctypes.c_int), ("k_lo", ctypes.c_int64), ("t_sft", ctypes.c_double),
                ("t0", ctypes.c_double), ("dtype", ctypes.c_int)]


class _BankDesc(ctypes.Structure):
    _fields_ = [("k0", ctypes.c_int64), ("n_f0", ctypes.c_int), ("n_f1", ctypes.c_int),
                ("f1", ctypes.c_void_p), ("n_sky", ctypes.c_int64), ("sky", ctypes.c_void_p),
                ("subband_bins", ctypes.c_int)]


class _BinaryDesc(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 6), ("hi", ctypes.c_double * 6), ("n_div", ctypes.c_int32 * 6),
                ("n_per_box", ctypes.c_int64), ("seed", ctypes.c_uint64)]


class _InjDesc(ctypes.Structure):
    _fields_ = [("k_sky", ctypes.c_int), ("half_f0", ctypes.c_int), ("half_window", ctypes.c_int),
                ("noise_scale", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("first_run_id", ctypes.c_uint64)]


# ft_injection {h0, cosi, psi, f0, f1, n[3]} and ft_inj_result {max_z, template_idx, n_oob}
INJECTION_DTYPE = np.dtype([("h0", "<f8"), ("cosi", "<f8"), ("psi", "<f8"), ("f0", "<f8"),
                            ("f1", "<f8"), ("n", "<f8", (3,))])
INJ_RESULT_DTYPE = np.dtype([("max_z", "<f8"), ("template_idx", "<i8"),
                             ("n_out_of_window", "<i8")])

_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64


def lib():
    """The loaded libfasttracks.so (raises FtError when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FtError(-6, f"{LIB_PATH} is not built (python -m paper_2411_18370_b300.build)")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "ft_last_error": (ctypes.c_char_p, []),
            "ft_abi_version": (_I, []),
            "ft_create": (_I, [ctypes.POINTER(_P), _I]),
            "ft_destroy": (None, [_P]),
            "ft_check_status": (_I, [_P, _P]),
            "ft_load_sfts": (_I, [_P, ctypes.POINTER(_BandDesc), _P, _I, _I64, _I, _P, _P, _P, _P,
                                  _P, ctypes.POINTER(_P)]),
            "ft_band_destroy": (None, [_P]),
            "ft_band_info": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                  ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]),
            "ft_make_bank": (_I, [_P, _P, ctypes.POINTER(_BankDesc), _P, ctypes.POINTER(_P)]),
            "ft_bank_destroy": (None, [_P]),
            "ft_bank_info": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
            "ft_required_wings": (_I, [ctypes.POINTER(_BandDesc), _P, _P, ctypes.POINTER(_BankDesc),
                                       ctypes.POINTER(_I), ctypes.POINTER(_I)]),
            "ft_eval_statistic": (_I, [_P, _P, _P, _P, _P, _P, _I, _P]),
            "ft_topk_per_band": (_I, [_P, _P, _P, _I, _P, _I, _P]),
            "ft_track_bins": (_I, [_P, _P, _P, _P, _I64, _P, _I, _P]),
            "ft_set_tune": (_I, [_P, _P]),
            "ft_gather_roof": (_I, [_P, _I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "ft_pdet_q": (_I, [_P, _P, _P, _I64, _P, _P, _P, _P]),
            "ft_band_set_sky_weights": (_I, [_P, _P, _P]),
            "ft_selftest_bounded_wait": (_I, [_P, ctypes.POINTER(ctypes.c_double), _P]),
            "ft_make_binary_bank": (_I, [_P, _P, ctypes.POINTER(_BinaryDesc), ctypes.POINTER(_P)]),
            "ft_binary_bank_destroy": (None, [_P]),
            "ft_binary_bank_info": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
            "ft_binary_templates": (_I, [_P, _P, _I64, _I64, _P, _P]),
            "ft_ctx_memory": (_I, [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
            "ft_binary_decisions": (_I, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]),
            "ft_binary_cos_screen_check": (_I, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "ft_binary_track_bins": (_I, [_P, _P, _P, _P, _I64, _P, _I, _P]),
            "ft_binary_eval": (_I, [_P, _P, _P, _I64, _I64, _P, _P, _P, _I, _P]),
            "ft_binary_topk_per_box": (_I, [_P, _P, _P, _I, _P, _I, _P]),
            "ft_binary_topk_per_box_gated": (_I, [_P, _P, _P, _I, _P, ctypes.c_float, _P, _I, _P]),
            "ft_number_count_band": (_I, [_P, _P, ctypes.c_double, _P, ctypes.POINTER(_P)]),
            "ft_topk_per_band_gated": (_I, [_P, _P, _P, _I, _P, ctypes.c_float, _P, _I, _P]),
            "ft_topk_per_skybox": (_I, [_P, _P, _P, _I, _I, _P, _I, _P]),
            "ft_topk_per_box": (_I, [_P, _P, _P, _I, _I, _I, _P, ctypes.c_float, _P, _I, _P]),
            "ft_bank_sky_order": (_I, [_P, _P]),
            "ft_topk_per_band_noalloc": (_I, [_P, _P, _P, _I, _P, _I, _P]),
            "ft_batch_create": (_I, [_P, _I, _P, _P, _I, _P, _P, ctypes.POINTER(_P)]),
            "ft_batch_run": (_I, [_P, _P, _I, _P]),
            "ft_batch_info": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P,
                                   ctypes.POINTER(_I)]),
            "ft_batch_destroy": (None, [_P]),
            "ft_eval_batched": (_I, [_P, _I, _P, _P, _I, _P, _I, _P, _P]),
            "ft_run_injections": (_I, [_P, _P, _P, _P, ctypes.POINTER(_InjDesc), _I64, _P, _P, _P]),
            "ft_mlp_create": (_I, [_P, _I, _I, ctypes.c_uint64, ctypes.POINTER(_P)]),
            "ft_mlp_destroy": (None, [_P]),
            "ft_mlp_n_params": (_I, [_P, ctypes.POINTER(_I64)]),
            "ft_mlp_get_params": (_I, [_P, _P]),
            "ft_mlp_set_params": (_I, [_P, _P]),
            "ft_mlp_get_state": (_I, [_P, _P, ctypes.POINTER(_I64)]),
            "ft_mlp_set_state": (_I, [_P, _P, _I64]),
            "ft_mlp_loss_grad": (_I, [_P, _P, _P, _I, _P, _P]),
            "ft_mlp_adam_step": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float]),
            "ft_mlp_train": (_I, [_P, _P, _P, _I64, _I, _I, ctypes.c_float, ctypes.c_uint64, _P]),
            "ft_mlp_predict": (_I, [_P, _P, _I64, _P, _I, _I, _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise FtError(rc, lib().ft_last_error().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device) of a numpy array or torch tensor; None -> (None, False)."""
    if x is None:
        return None, False
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), bool(x.is_cuda)
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data, False


def _nbytes(x):
    if _is_torch(x):
        return x.numel() * x.element_size()
    return int(x.nbytes)


def _need(x, n_bytes, what):
    """Raise ValueError unless buffer x holds at least n_bytes (the library writes that many)."""
    if x is None:
        return
    if _nbytes(x) < n_bytes:
        raise ValueError(f"{what}: buffer of {_nbytes(x)} bytes, the call writes {n_bytes}")


def _gate_ptr(gate, n_templates, what):
    """Device pointer of a gate: a contiguous CUDA float32 tensor of n_templates values."""
    pg, gdev = _ptr(gate)
    if not gdev:
        raise ValueError(f"{what}: gate must be a CUDA tensor")
    if str(gate.dtype) != "torch.float32":
        raise ValueError(f"{what}: gate must be float32")
    if gate.numel() != n_templates:
        raise ValueError(f"{what}: gate has {gate.numel()} values, the bank {n_templates} templates")
    return pg


def _stream(stream, on_device):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    if on_device:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Context:
    def __init__(self, device: int = 0):
        h = _P()
        _check(lib().ft_create(ctypes.byref(h), device))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().ft_destroy(self.handle)
            self.handle = None

    def memory(self):
        """ft_ctx_memory: (scratch bytes, staging bytes) the context holds on its device."""
        a, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
        _check(lib().ft_ctx_memory(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def check_status(self, stream=None):
        _check(lib().ft_check_status(self.handle, _stream(stream, True)))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Band:
    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.handle = handle
        n, w, st, dt = _I64(), _I(), _I(), _I()
        mu, sg = ctypes.c_double(), ctypes.c_double()
        _check(lib().ft_band_info(handle, ctypes.byref(n), ctypes.byref(w), ctypes.byref(st),
                                  ctypes.byref(dt), ctypes.byref(mu), ctypes.byref(sg)))
        self.n_sft, self.n_bins, self.row_stride, self.dtype = n.value, w.value, st.value, dt.value
        self.mu_g, self.sigma_g = mu.value, sg.value

    def close(self):
        if self.handle:
            lib().ft_band_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Bank:
    def __init__(self, band, handle):
        self.band = band
        self.handle = handle
        nt, ns, ws = _I64(), _I(), _I()
        _check(lib().ft_bank_info(handle, ctypes.byref(nt), ctypes.byref(ns), ctypes.byref(ws)))
        self.n_templates, self.n_subbands, self.window_safe = nt.value, ns.value, bool(ws.value)

    def close(self):
        if self.handle:
            lib().ft_bank_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Tune(ctypes.Structure):
    _fields_ = [("rows_per_stage", ctypes.c_int), ("stages", ctypes.c_int), ("tile_f0", ctypes.c_int)]


def band_set_sky_weights(band, det_tensor, stream=None):
    """ft_band_set_sky_weights: turn on the all-sky weights (a^2 + b^2) / S_n of Sec. II.B
    for banks made from now on (det_tensor [N_SFT][6]), or off again with None."""
    if det_tensor is None:
        _check(lib().ft_band_set_sky_weights(band.handle, None, _stream(stream, False)))
        return
    D = np.ascontiguousarray(det_tensor, np.float64)
    if D.shape != (band.n_sft, 6):
        raise ValueError("det_tensor must be [N_SFT][6]")
    _check(lib().ft_band_set_sky_weights(band.handle, D.ctypes.data, _stream(stream, False)))


class BinaryBank:
    """A random binary-orbit bank in hyperboxes (ft_make_binary_bank)."""

    def __init__(self, band, handle):
        self.band = band
        self.handle = handle
        nt, nb = _I64(), _I64()
        _check(lib().ft_binary_bank_info(handle, ctypes.byref(nt), ctypes.byref(nb)))
        self.n_templates, self.n_boxes = nt.value, nb.value

    def close(self):
        if self.handle:
            lib().ft_binary_bank_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_binary_bank(ctx, band, lo, hi, n_div, n_per_box, seed) -> BinaryBank:
    """ft_make_binary_bank: lo / hi per dimension (f0 Hz, alpha turns, sin(delta), a_p
    light-seconds, Omega rad/s, phi_b turns), n_div boxes per dimension, n_per_box templates
    per box, Philox seed."""
    d = _BinaryDesc()
    for k in range(6):
        d.lo[k] = float(lo[k])
        d.hi[k] = float(hi[k])
        d.n_div[k] = int(n_div[k])
    d.n_per_box = int(n_per_box)
    d.seed = int(seed) & ((1 << 64) - 1)
    h = _P()
    _check(lib().ft_make_binary_bank(ctx.handle, band.handle, ctypes.byref(d), ctypes.byref(h)))
    return BinaryBank(band, h)


def binary_decisions(bank):
    """ft_binary_decisions: (FP64 decisions since the last call, the bank's screening bound
    delta in bins); resets the count."""
    n = ctypes.c_uint64(0)
    d = ctypes.c_double(0.0)
    _check(lib().ft_binary_decisions(bank.handle, ctypes.byref(n), ctypes.byref(d)))
    return int(n.value), float(d.value)


def binary_cos_screen_check(ctx):
    """ft_binary_cos_screen_check: (largest error of the binary screen's cosine step over all
    2^32 orbit phases, the bound the screen's delta assumes)."""
    m = ctypes.c_double(0.0)
    bnd = ctypes.c_double(0.0)
    _check(lib().ft_binary_cos_screen_check(ctx.handle, ctypes.byref(m), ctypes.byref(bnd)))
    return float(m.value), float(bnd.value)


def binary_templates(ctx, bank, first, n, stream=None):
    """lambda [n][6] of templates first .. first + n - 1 as the kernels derive them."""
    out = np.empty((int(n), 6), np.float64)
    _check(lib().ft_binary_templates(ctx.handle, bank.handle, int(first), int(n), out.ctypes.data,
                                     _stream(stream, False)))
    return out


def binary_track_bins(ctx, band, bank, templates, out, stream=None):
    """ft_binary_track_bins: templates int64 [n], out int32 [n, N_SFT]; both host or device."""
    pt, dev = _ptr(templates)
    pb, dev2 = _ptr(out)
    if dev != dev2:
        raise ValueError("templates and out must both be host or both device")
    if str(templates.dtype) not in ("int64", "torch.int64"):
        raise ValueError("binary_track_bins: templates must be int64")
    _need(out, 4 * int(templates.shape[0]) * band.n_sft, "binary_track_bins out")
    _check(lib().ft_binary_track_bins(ctx.handle, band.handle, bank.handle, pt, int(templates.shape[0]),
                                      pb, int(dev), _stream(stream, dev)))


def binary_eval(ctx, band, bank, first, n, s_out, z_out=None, n_oob_out=None, stream=None):
    """ft_binary_eval: s (and z, out-of-window counts) of templates first .. first + n - 1."""
    for x, nm in ((s_out, "s_out"), (z_out, "z_out"), (n_oob_out, "n_oob_out")):
        _need(x, 4 * max(int(n), 0), f"binary_eval {nm}")
    ps, dev = _ptr(s_out)
    pz, _ = _ptr(z_out)
    po, _ = _ptr(n_oob_out)
    _check(lib().ft_binary_eval(ctx.handle, band.handle, bank.handle, int(first), int(n), ps, pz, po,
                                int(dev), _stream(stream, dev)))


def binary_topk_per_box(ctx, band, bank, k, out, stream=None):
    """ft_binary_topk_per_box into a CANDIDATE_DTYPE [n_boxes, k] array or a device byte
    tensor of n_boxes * k * 16 bytes."""
    _need(out, bank.n_boxes * int(k) * 16, "binary_topk_per_box out")
    po, dev = _ptr(out)
    _check(lib().ft_binary_topk_per_box(ctx.handle, band.handle, bank.handle, int(k), po, int(dev),
                                        _stream(stream, dev)))


def binary_topk_per_box_gated(ctx, band, bank, k, gate, gate_min, out, stream=None):
    """ft_binary_topk_per_box_gated: gate is a CUDA float32 tensor of n_templates values."""
    pg = _gate_ptr(gate, bank.n_templates, "binary_topk_per_box_gated")
    _need(out, bank.n_boxes * int(k) * 16, "binary_topk_per_box_gated out")
    po, dev = _ptr(out)
    _check(lib().ft_binary_topk_per_box_gated(ctx.handle, band.handle, bank.handle, int(k), pg,
                                              float(gate_min), po, int(dev), _stream(stream, dev)))


def number_count_band(ctx, band, threshold=3.2, stream=None):
    """ft_number_count_band: a band holding 1[P > threshold] (Eq. (number_count)) with the
    source band's weights; its mu_g / sigma_g are the weighted count's noise moments."""
    h = _P()
    _check(lib().ft_number_count_band(ctx.handle, band.handle, float(threshold),
                                      _stream(stream, False), ctypes.byref(h)))
    return Band(ctx, h)


def pdet_q(ctx, band, det_tensor, pop, stream=None):
    """ft_pdet_q: per population draw (INJECTION_DTYPE records; h0, f0, f1 unused) the sums
    (w rho^2, w^2 rho^2) over the band's SFTs at h0 = 1 (Sec. V.A)."""
    pop = np.ascontiguousarray(pop, dtype=INJECTION_DTYPE)
    D = np.ascontiguousarray(det_tensor, np.float64).reshape(-1, 6)
    if len(D) != band.n_sft:
        raise ValueError("det_tensor must be [N_SFT][6]")
    n = len(pop)
    r1 = np.empty(n, np.float64)
    r2 = np.empty(n, np.float64)
    _check(lib().ft_pdet_q(ctx.handle, band.handle, D.ctypes.data, n, pop.ctypes.data,
                           r1.ctypes.data, r2.ctypes.data, _stream(stream, False)))
    return r1, r2


def selftest_bounded_wait(ctx, stream=None):
    """ft_selftest_bounded_wait: returns (return code, seconds waited on the device); the code
    is FT_ERR_TIMEOUT when the bounded wait and the status plumbing work."""
    w = ctypes.c_double()
    rc = lib().ft_selftest_bounded_wait(ctx.handle, ctypes.byref(w), _stream(stream, False))
    return rc, w.value


def gather_roof(ctx, dtype="f16"):
    """ft_gather_roof: measured evaluations/s and evaluations/clock/SM of the bare
    gather-accumulate loop for a storage type."""
    e = ctypes.c_double()
    c = ctypes.c_double()
    _check(lib().ft_gather_roof(ctx.handle, DTYPES[dtype], ctypes.byref(e), ctypes.byref(c)))
    return e.value, c.value


def set_tune(ctx, rows_per_stage=0, stages=0, tile_f0=0):
    """ft_set_tune: launch-shape override for later calls on ctx (all zeros clears it)."""
    if rows_per_stage == stages == tile_f0 == 0:
        _check(lib().ft_set_tune(ctx.handle, None))
        return
    t = _Tune(int(rows_per_stage), int(stages), int(tile_f0))
    _check(lib().ft_set_tune(ctx.handle, ctypes.byref(t)))


class Batch:
    """ft_batch: many (band, bank) pairs searched by one graph-captured persistent launch."""

    def __init__(self, ctx, bands, banks, k, tile_f0=0, stages=0, stream=None):
        n = len(bands)
        self.ctx, self.bands, self.banks, self.k = ctx, list(bands), list(banks), int(k)
        barr = (_P * n)(*[b.handle for b in bands])
        karr = (_P * n)(*[b.handle for b in banks])
        tune = None
        if tile_f0 or stages:
            tune = ctypes.byref(_Tune(0, int(stages), int(tile_f0)))
        h = _P()
        _check(lib().ft_batch_create(ctx.handle, n, barr, karr, self.k, tune,
                                     _stream(stream, False), ctypes.byref(h)))
        self.handle = h
        nc, ev, nct = _I64(), _I64(), _I()
        t = _Tune()
        _check(lib().ft_batch_info(h, ctypes.byref(nc), ctypes.byref(ev), ctypes.byref(t),
                                   ctypes.byref(nct)))
        self.n_candidates, self.evals, self.n_ctas = nc.value, ev.value, nct.value
        self.tile_f0, self.stages, self.rows_per_stage = t.tile_f0, t.stages, t.rows_per_stage
        self.n_subbands = [b.n_subbands for b in banks]

    def run(self, out, stream=None):
        po, dev = _ptr(out)
        _check(lib().ft_batch_run(self.handle, po, int(dev), _stream(stream, dev)))

    def close(self):
        if self.handle:
            lib().ft_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_injections(ctx, band, bank, det_tensor, inj, seed, first_run_id=0, k_sky=64, half_f0=2,
                   half_window=160, noise_scale=1.0, stream=None):
    """ft_run_injections: one injection-recovery run per record of `inj` (INJECTION_DTYPE);
    returns an INJ_RESULT_DTYPE array (max z over the local bank, its template, reads outside
    the generated window)."""
    arr = np.ascontiguousarray(inj, dtype=INJECTION_DTYPE)
    D = _f64(det_tensor).reshape(-1, 6)
    if len(D) != band.n_sft:
        raise ValueError("det_tensor must be [N_SFT][6]")
    out = np.zeros(len(arr), dtype=INJ_RESULT_DTYPE)
    d = _InjDesc(int(k_sky), int(half_f0), int(half_window), float(noise_scale), int(seed),
                 int(first_run_id))
    _check(lib().ft_run_injections(ctx.handle, band.handle, bank.handle, D.ctypes.data,
                                   ctypes.byref(d), len(arr), arr.ctypes.data, out.ctypes.data,
                                   _stream(stream, False)))
    return out


class MLP:
    """ft_mlp: the p_det surrogate network (4 layers, ReLU, sigmoid output)."""

    def __init__(self, ctx, d_in, width=128, seed=0):
        h = _P()
        _check(lib().ft_mlp_create(ctx.handle, int(d_in), int(width), int(seed), ctypes.byref(h)))
        self.ctx, self.handle, self.d_in, self.width = ctx, h, int(d_in), int(width)
        n = _I64()
        _check(lib().ft_mlp_n_params(h, ctypes.byref(n)))
        self.n_params = n.value

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        _check(lib().ft_mlp_get_params(self.handle, out.ctypes.data))
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        assert th.size == self.n_params
        _check(lib().ft_mlp_set_params(self.handle, th.ctypes.data))

    def get_state(self):
        """(state [3, n_params]: parameters, Adam moments m and v; Adam step count)."""
        st = np.empty((3, self.n_params), np.float32)
        t = _I64()
        _check(lib().ft_mlp_get_state(self.handle, st.ctypes.data, ctypes.byref(t)))
        return st, t.value

    def set_state(self, state, adam_t):
        st = np.ascontiguousarray(state, dtype=np.float32)
        assert st.shape == (3, self.n_params)
        _check(lib().ft_mlp_set_state(self.handle, st.ctypes.data, int(adam_t)))

    def loss_grad(self, X, y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        loss = ctypes.c_float()
        g = np.empty(self.n_params, np.float32)
        _check(lib().ft_mlp_loss_grad(self.handle, X.ctypes.data, y.ctypes.data, len(y),
                                      ctypes.byref(loss), g.ctypes.data))
        return loss.value, g

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().ft_mlp_adam_step(self.handle, lr, beta1, beta2, eps))

    def train(self, X, y, batch=1024, epochs=10, lr=1e-3, seed=0):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        hist = np.empty(max(epochs, 1), np.float32)
        _check(lib().ft_mlp_train(self.handle, X.ctypes.data, y.ctypes.data, len(y), int(batch),
                                  int(epochs), float(lr), int(seed), hist.ctypes.data))
        return hist[:epochs]

    def predict(self, X, bf16=True, tensor_cores=True):
        """ft_mlp_predict: p for the rows of X.  bf16: BF16 inference (on the tensor cores
        unless tensor_cores is False), else the FP32 forward."""
        mode = 0 if not bf16 else (1 if tensor_cores else 2)
        if _is_torch(X) and X.is_cuda:
            import torch

            p = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
            _check(lib().ft_mlp_predict(self.handle, X.data_ptr(), X.shape[0], p.data_ptr(),
                                        mode, 1, _stream(None, True)))
            return p
        X = np.ascontiguousarray(X, dtype=np.float32)
        p = np.empty(len(X), np.float32)
        _check(lib().ft_mlp_predict(self.handle, X.ctypes.data, len(X), p.ctypes.data, mode,
                                    0, None))
        return p

    def close(self):
        if self.handle:
            lib().ft_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def abi_version() -> int:
    return lib().ft_abi_version()


def create(device: int = 0) -> Context:
    return Context(device)


def _band_desc(n_sft, n_bins, k_lo, t_sft, t0, dtype):
    arr = (ctypes.c_int * len(n_sft))(*[int(x) for x in n_sft])
    d = _BandDesc(len(n_sft), arr, int(n_bins), int(k_lo), float(t_sft), float(t0),
                  DTYPES[dtype] if isinstance(dtype, str) else int(dtype))
    return d, arr


def _bank_desc(k0, n_f0, f1, sky, subband_bins):
    f1 = _f64(f1)
    sky = _f64(sky).reshape(-1, 3)
    d = _BankDesc(int(k0), int(n_f0), len(f1), f1.ctypes.data, len(sky), sky.ctypes.data,
                  int(subband_bins))
    return d, (f1, sky)


def load_sfts(ctx, power, t_mid, v_over_c, n_sft, k_lo, t_sft, t0, dtype="f32", w=None,
              s_n=None, n_bins=None, stream=None) -> Band:
    """ft_load_sfts: power [N, stride] float32/float64 (numpy or torch, host or device)."""
    if _is_torch(power):
        import torch

        pdt = {torch.float32: FT_F32, torch.float64: FT_F64}[power.dtype]
    else:
        power = np.ascontiguousarray(power)
        pdt = {np.dtype(np.float32): FT_F32, np.dtype(np.float64): FT_F64}[power.dtype]
    stride = int(power.shape[1])
    n_bins = stride if n_bins is None else int(n_bins)
    desc, keep = _band_desc(n_sft, n_bins, k_lo, t_sft, t0, dtype)
    pp, on_dev = _ptr(power)
    t_mid = _f64(t_mid)
    v = _f64(v_over_c).reshape(-1, 3)
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    sn = None if s_n is None else _f64(s_n)
    # the ABI takes arrays of N_SFT = sum(n_sft) entries: check the lengths here
    N = int(np.sum(np.asarray(n_sft, np.int64)))
    if (int(power.shape[0]) != N or len(t_mid) != N or len(v) != N or (wv is not None and len(wv) != N)
            or (sn is not None and len(sn) != N)):
        raise ValueError("power rows, t_mid, v_over_c, w and s_n must all have sum(n_sft) entries")
    h = _P()
    _check(lib().ft_load_sfts(ctx.handle, ctypes.byref(desc), pp, pdt, stride, int(on_dev),
                              t_mid.ctypes.data, v.ctypes.data,
                              None if wv is None else wv.ctypes.data,
                              None if sn is None else sn.ctypes.data,
                              _stream(stream, on_dev), ctypes.byref(h)))
    return Band(ctx, h)


def make_bank(ctx, band, k0, n_f0, f1, sky, subband_bins, stream=None) -> Bank:
    desc, keep = _bank_desc(k0, n_f0, f1, sky, subband_bins)
    h = _P()
    _check(lib().ft_make_bank(ctx.handle, band.handle, ctypes.byref(desc), _stream(stream, False),
                              ctypes.byref(h)))
    b = Bank(band, h)
    b.n_f0, b.n_f1, b.n_sky = int(desc.n_f0), int(desc.n_f1), int(desc.n_sky)
    return b


def required_wings(n_sft, t_mid, v_over_c, t_sft, t0, k0, n_f0, f1, sky, subband_bins=1):
    bd, keep1 = _band_desc(n_sft, 1, 0, t_sft, t0, "f32")
    kd, keep2 = _bank_desc(k0, n_f0, f1, sky, subband_bins)
    t_mid = _f64(t_mid)
    v = _f64(v_over_c).reshape(-1, 3)
    lo, hi = _I(), _I()
    _check(lib().ft_required_wings(ctypes.byref(bd), t_mid.ctypes.data, v.ctypes.data,
                                   ctypes.byref(kd), ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def eval_statistic(ctx, band, bank, s_out, z_out=None, n_oob_out=None, stream=None):
    """ft_eval_statistic into caller-owned float32 s_out (and z_out, int32 n_oob_out)."""
    for x, nm in ((s_out, "s_out"), (z_out, "z_out"), (n_oob_out, "n_oob_out")):
        _need(x, 4 * bank.n_templates, f"eval_statistic {nm}")
    ps, dev = _ptr(s_out)
    pz, _ = _ptr(z_out)
    po, _ = _ptr(n_oob_out)
    _check(lib().ft_eval_statistic(ctx.handle, band.handle, bank.handle, ps, pz, po, int(dev),
                                   _stream(stream, dev)))


def topk_per_band(ctx, band, bank, k, out, stream=None):
    """ft_topk_per_band into `out`: a host numpy array of CANDIDATE_DTYPE [n_sub, k] or a
    device byte tensor of n_sub * k * 16 bytes (decode with decode_candidates)."""
    _need(out, bank.n_subbands * int(k) * 16, "topk_per_band out")
    po, dev = _ptr(out)
    _check(lib().ft_topk_per_band(ctx.handle, band.handle, bank.handle, int(k), po, int(dev),
                                  _stream(stream, dev)))


def topk_per_band_gated(ctx, band, bank, k, gate, gate_min, out, stream=None):
    """ft_topk_per_band_gated: as topk_per_band over the templates with gate[t] >= gate_min;
    gate is a CUDA float32 tensor of n_templates values (e.g. the weighted number count)."""
    pg = _gate_ptr(gate, bank.n_templates, "topk_per_band_gated")
    _need(out, bank.n_subbands * int(k) * 16, "topk_per_band_gated out")
    po, dev = _ptr(out)
    _check(lib().ft_topk_per_band_gated(ctx.handle, band.handle, bank.handle, int(k), pg,
                                        float(gate_min), po, int(dev), _stream(stream, dev)))


def topk_per_skybox(ctx, band, bank, sky_box, k, out, stream=None):
    """ft_topk_per_skybox into `out` (CANDIDATE_DTYPE [n_sky_boxes, n_sub, k] host array or a
    device byte tensor)."""
    if int(sky_box) >= 1:
        _need(out, -(-bank.n_sky // int(sky_box)) * bank.n_subbands * int(k) * 16, "topk_per_skybox out")
    po, dev = _ptr(out)
    _check(lib().ft_topk_per_skybox(ctx.handle, band.handle, bank.handle, int(sky_box), int(k), po,
                                    int(dev), _stream(stream, dev)))


def topk_per_box(ctx, band, bank, sky_box, f1_box, k, out, gate=None, gate_min=0.0, stream=None):
    """ft_topk_per_box into `out` (CANDIDATE_DTYPE [n_sky_boxes, n_f1_boxes, n_sub, k] host
    array or a device byte tensor); gate: None, or a CUDA float32 tensor of n_templates values
    as in topk_per_band_gated."""
    pg = None
    if gate is not None:
        pg = _gate_ptr(gate, bank.n_templates, "topk_per_box")
    if int(sky_box) >= 1 and int(f1_box) >= 1:
        nb = -(-bank.n_sky // int(sky_box)) * -(-bank.n_f1 // int(f1_box))
        _need(out, nb * bank.n_subbands * int(k) * 16, "topk_per_box out")
    po, dev = _ptr(out)
    _check(lib().ft_topk_per_box(ctx.handle, band.handle, bank.handle, int(sky_box), int(f1_box),
                                 int(k), pg, float(gate_min), po, int(dev), _stream(stream, dev)))


def bank_sky_order(bank, n_sky=None):
    """ft_bank_sky_order: the bank's sky order (int32 [n_sky]); n_sky, when given, must be the
    bank's."""
    if n_sky is not None and int(n_sky) != bank.n_sky:
        raise ValueError(f"bank_sky_order: the bank has {bank.n_sky} sky points, not {n_sky}")
    out = np.empty(bank.n_sky, np.int32)
    _check(lib().ft_bank_sky_order(bank.handle, out.ctypes.data))
    return out


def topk_per_band_noalloc(ctx, band, bank, k, out, stream=None):
    """ft_topk_per_band_noalloc: as topk_per_band, with the candidate scratch in the
    library's fixed device array instead of memory allocated during the call."""
    _need(out, bank.n_subbands * int(k) * 16, "topk_per_band_noalloc out")
    po, dev = _ptr(out)
    _check(lib().ft_topk_per_band_noalloc(ctx.handle, band.handle, bank.handle, int(k), po,
                                          int(dev), _stream(stream, dev)))


def decode_candidates(buf, n_sub, k):
    """(template_idx int64 [n_sub, k], s float32, z float32) from a candidate buffer."""
    if _is_torch(buf):
        buf = buf.cpu().numpy()
    arr = np.frombuffer(np.ascontiguousarray(buf).tobytes(), dtype=CANDIDATE_DTYPE).reshape(n_sub, k)
    return arr["template_idx"].copy(), arr["s"].copy(), arr["z"].copy()


def track_bins(ctx, band, bank, templates, out, stream=None):
    """ft_track_bins: templates int64 [n], out int32 [n, N_SFT]; both host or both device."""
    pt, dev = _ptr(templates)
    pb, dev2 = _ptr(out)
    if dev != dev2:
        raise ValueError("templates and out must both be host or both device")
    n = templates.shape[0]
    if str(templates.dtype) not in ("int64", "torch.int64"):
        raise ValueError("track_bins: templates must be int64")
    _need(out, 4 * n * band.n_sft, "track_bins out")
    _check(lib().ft_track_bins(ctx.handle, band.handle, bank.handle, pt, n, pb, int(dev),
                               _stream(stream, dev)))

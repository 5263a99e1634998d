"""Thin ctypes binding of libdmpt.so (the C ABI in include/dmpt.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch provides device memory and the stream.  If the library is
missing the binding raises; there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdmpt.so")

DMPT_MAX_K = 8
DMPT_MAX_LAYERS = 256

PRECISIONS = {"fp64": 0, "fp32": 1, "dual_fp16": 2, "dual_bf16": 3}

STATUS = {
    0: "DMPT_OK", 1: "DMPT_EINVAL", 2: "DMPT_EWORKSPACE", 3: "DMPT_ENOTCONV",
    4: "DMPT_ENUMERIC", 5: "DMPT_ETIMEOUT", 6: "DMPT_ECUDA", 7: "DMPT_EUNSUPPORTED",
}


class DmptOptions(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("max_layers", ctypes.c_int),
        ("c_pt", ctypes.c_double),
        ("c_d0", ctypes.c_double),
        ("operand_scaling", ctypes.c_int),
        ("sync_every", ctypes.c_int),
        ("timing", ctypes.c_int),
        ("timeout_s", ctypes.c_double),
        ("ckpt_every", ctypes.c_int),
        ("accum_chunk", ctypes.c_int),
        ("cta_pair", ctypes.c_int),
        ("k_snake", ctypes.c_int),
        ("order", ctypes.c_int),
        ("tile_band", ctypes.c_int),
        ("inject_stall", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("round_align", ctypes.c_int),
        ("hole_form", ctypes.c_int),
        ("group_tile_n", ctypes.c_int),
    ]


class DmptInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("layers", ctypes.c_int),
        ("d0_layer", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("d1_layer", ctypes.c_int * DMPT_MAX_K),
        ("eps_min", ctypes.c_double),
        ("eps_max", ctypes.c_double),
        ("froerr0", ctypes.c_double),
        ("froerr1", ctypes.c_double * DMPT_MAX_K),
        ("ms_layers", ctypes.c_double),
        ("product_launches", ctypes.c_int),
        ("timed_launches", ctypes.c_int),
        ("mma_flops", ctypes.c_double),
        ("alg_flops", ctypes.c_double),
        ("sigma", ctypes.c_byte * DMPT_MAX_LAYERS),
        ("n_s", ctypes.c_double * DMPT_MAX_LAYERS),
        ("n_x", ctypes.c_double * DMPT_MAX_LAYERS),
        ("iderr", ctypes.c_double * DMPT_MAX_LAYERS),
        ("froerr1_hist", (ctypes.c_double * DMPT_MAX_LAYERS) * DMPT_MAX_K),
        ("hole", ctypes.c_int),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdmpt.so and declare its exported functions."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run __graft_entry__.build() "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.dmpt_create.argtypes = [ctypes.POINTER(vp), c_int]
    lib.dmpt_create.restype = c_int
    lib.dmpt_destroy.argtypes = [vp]
    lib.dmpt_destroy.restype = c_int
    lib.dmpt_default_options.argtypes = [ctypes.POINTER(DmptOptions)]
    lib.dmpt_default_options.restype = None
    lib.dmpt_status_string.argtypes = [c_int]
    lib.dmpt_status_string.restype = ctypes.c_char_p
    lib.dmpt_last_error.argtypes = [vp]
    lib.dmpt_last_error.restype = ctypes.c_char_p
    lib.dmpt_workspace_size.argtypes = [i64, c_int, ctypes.POINTER(DmptOptions)]
    lib.dmpt_workspace_size.restype = ctypes.c_size_t
    lib.dmpt_bounds.argtypes = [vp, vp, i64, i64, vp, vp]
    lib.dmpt_bounds.restype = c_int
    lib.dmpt_sp2_response.argtypes = [vp, vp, vp, c_int, i64, i64, i64,
                                      ctypes.POINTER(DmptOptions), vp, vp,
                                      ctypes.POINTER(DmptInfo), vp, ctypes.c_size_t, vp]
    lib.dmpt_sp2_response.restype = c_int
    lib.dmpt_sp2_response2.argtypes = [vp, vp, vp, c_int, i64, i64, i64,
                                       ctypes.POINTER(DmptOptions), vp, vp, vp,
                                       ctypes.POINTER(DmptInfo), vp, ctypes.c_size_t, vp]
    lib.dmpt_sp2_response2.restype = c_int
    lib.dmpt_sp2_response_m.argtypes = [vp, vp, vp, c_int, i64, i64, i64, c_int,
                                        ctypes.POINTER(DmptOptions), vp, vp, vp,
                                        ctypes.POINTER(DmptInfo), vp, ctypes.c_size_t, vp]
    lib.dmpt_sp2_response_m.restype = c_int
    lib.dmpt_sp2_backward.argtypes = [vp, vp, i64, i64, ctypes.POINTER(DmptOptions), vp, vp,
                                      ctypes.c_size_t, vp]
    lib.dmpt_sp2_backward.restype = c_int
    lib.dmpt_response_replay.argtypes = [vp, vp, c_int, i64, i64, ctypes.POINTER(DmptOptions),
                                         vp, ctypes.POINTER(DmptInfo), vp, ctypes.c_size_t, vp]
    lib.dmpt_response_replay.restype = c_int
    lib.dmpt_scc_response.argtypes = [vp, vp, vp, c_int, i64, i64, ctypes.POINTER(DmptOptions),
                                      ctypes.c_double, c_int, ctypes.c_double, vp,
                                      ctypes.POINTER(DmptInfo), ctypes.POINTER(c_int),
                                      ctypes.POINTER(ctypes.c_double), vp, ctypes.c_size_t, vp]
    lib.dmpt_scc_response.restype = c_int
    lib.dmpt_autotune.argtypes = [vp, vp, vp, c_int, i64, i64, i64, ctypes.POINTER(DmptOptions),
                                  c_int, vp, vp, ctypes.POINTER(DmptOptions),
                                  ctypes.POINTER(ctypes.c_double), vp, ctypes.c_size_t, vp]
    lib.dmpt_autotune.restype = c_int
    lib.dmpt_workspace_size_host.argtypes = [i64, c_int, ctypes.POINTER(DmptOptions)]
    lib.dmpt_workspace_size_host.restype = ctypes.c_size_t
    lib.dmpt_host_copy_in_bytes.argtypes = [i64, c_int]
    lib.dmpt_host_copy_in_bytes.restype = ctypes.c_size_t
    lib.dmpt_sp2_response_host.argtypes = [vp, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int,
                                           i64, i64, ctypes.POINTER(DmptOptions),
                                           ctypes.POINTER(vp), ctypes.POINTER(vp),
                                           ctypes.POINTER(DmptInfo), vp, ctypes.c_size_t, vp]
    lib.dmpt_sp2_response_host.restype = c_int
    lib.dmpt_workspace_size_batch.argtypes = [c_int, ctypes.POINTER(i64), c_int,
                                              ctypes.POINTER(DmptOptions)]
    lib.dmpt_workspace_size_batch.restype = ctypes.c_size_t
    lib.dmpt_sp2_response_batch.argtypes = [vp, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), c_int,
                                            ctypes.POINTER(i64), ctypes.POINTER(i64),
                                            ctypes.POINTER(i64), ctypes.POINTER(DmptOptions),
                                            ctypes.POINTER(vp), ctypes.POINTER(vp),
                                            ctypes.POINTER(DmptInfo), vp, ctypes.c_size_t, vp]
    lib.dmpt_sp2_response_batch.restype = c_int
    lib.dmpt_sp2_response_static.argtypes = [vp, vp, vp, c_int, i64, i64, i64,
                                             ctypes.POINTER(DmptOptions), vp, vp,
                                             ctypes.POINTER(DmptInfo), vp]
    lib.dmpt_sp2_response_static.restype = c_int
    _lib = lib
    return lib


class DmptError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


@dataclass
class Info:
    status: int
    layers: int
    d0_layer: int
    converged: bool
    d1_layer: list
    eps_min: float
    eps_max: float
    froerr0: float
    froerr1: list
    ms_layers: float
    product_launches: int
    timed_launches: int
    mma_flops: float
    alg_flops: float
    sigma: list
    # per-layer stopping quantities (index n - 1 = layer n): N_S, N_X, IdErr of
    # Alg. 2 up to d0_layer; FroErr^(1) of Alg. 3 per slot up to `layers`
    n_s: list = None
    n_x: list = None
    iderr: list = None
    froerr1_hist: list = None
    hole: bool = False

    @classmethod
    def from_c(cls, ci: DmptInfo, k: int) -> "Info":
        d0 = ci.d0_layer if ci.d0_layer > 0 else ci.layers
        return cls(status=ci.status, layers=ci.layers, d0_layer=ci.d0_layer,
                   converged=bool(ci.converged), d1_layer=list(ci.d1_layer[:k]),
                   eps_min=ci.eps_min, eps_max=ci.eps_max, froerr0=ci.froerr0,
                   froerr1=list(ci.froerr1[:k]), ms_layers=ci.ms_layers,
                   product_launches=ci.product_launches, timed_launches=ci.timed_launches,
                   mma_flops=ci.mma_flops, alg_flops=ci.alg_flops,
                   sigma=list(ci.sigma[:ci.layers]), n_s=list(ci.n_s[:d0]),
                   n_x=list(ci.n_x[:d0]), iderr=list(ci.iderr[:d0]),
                   froerr1_hist=[list(ci.froerr1_hist[j][:ci.layers]) for j in range(k)],
                   hole=bool(ci.hole))


def options(precision="dual_fp16", max_layers=100, c_pt=9.0, c_d0=4.5, operand_scaling=1,
            sync_every=4, timing=False, timeout_s=2.0, accum_chunk=0,
            cta_pair=1, k_snake=1, ckpt_every=0, order=1, tile_band=8,
            inject_stall=0, autotune=0, round_align=1, hole_form=1,
            group_tile_n=256) -> DmptOptions:
    lib = load_library()
    o = DmptOptions()
    lib.dmpt_default_options(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.max_layers = int(max_layers)
    o.c_pt = float(c_pt)
    o.c_d0 = float(c_d0)
    o.operand_scaling = int(operand_scaling)
    o.sync_every = int(sync_every)
    o.timing = int(bool(timing))
    o.timeout_s = float(timeout_s)
    o.accum_chunk = int(accum_chunk)
    o.cta_pair = int(cta_pair)
    o.k_snake = int(k_snake)
    o.ckpt_every = int(ckpt_every)
    o.order = int(order)
    o.tile_band = int(tile_band)
    o.inject_stall = int(inject_stall)
    o.autotune = int(autotune)
    o.round_align = int(round_align)
    o.hole_form = int(hole_form)
    o.group_tile_n = int(group_tile_n)
    return o


class Context:
    """A dmpt handle on one CUDA device plus a cached workspace tensor."""

    def __init__(self, device: int = 0):
        import torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("dmpt needs a CUDA device (GB300, sm_103a)")
        self.device = device
        h = ctypes.c_void_p()
        st = self.lib.dmpt_create(ctypes.byref(h), device)
        if st != 0:
            raise DmptError(st, self.lib.dmpt_status_string(st).decode())
        self.h = h
        self._ws = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmpt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise DmptError(st, self.lib.dmpt_last_error(self.h).decode())

    def workspace_size(self, n: int, k: int, opts: DmptOptions) -> int:
        return int(self.lib.dmpt_workspace_size(n, k, ctypes.byref(opts)))

    def workspace(self, nbytes: int):
        import torch
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = None
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
        ptr = self._ws.data_ptr()
        off = (-ptr) % 256
        return ptr + off, self._ws.numel() - off

    def bounds(self, H, stream=None):
        """Gershgorin (eps_1, eps_N) of a float64 CUDA matrix H, as a 2-element tensor."""
        import torch
        n = H.shape[0]
        eps = torch.empty(2, dtype=torch.float64, device=H.device)
        s = stream if stream is not None else torch.cuda.current_stream(H.device)
        self._check(self.lib.dmpt_bounds(self.h, H.data_ptr(), n, H.stride(0), eps.data_ptr(),
                                         ctypes.c_void_p(s.cuda_stream)))
        return eps

    def sp2_response(self, H, H1, n_occ: int, precision="dual_fp16", out=None,
                     want_P=True, stream=None, raise_on_error=True, workspace=None, **kw):
        """P and P1 of (H, H1) by DNN-SP2-PT on the device.

        H: (n, n) float64 CUDA tensor; H1: (n, n), (k, n, n) or None (P only).
        Returns (P or None, P1 of shape (k, n, n) or None, Info).  `workspace`
        (a uint8 CUDA tensor) overrides the context's shared workspace.
        """
        import torch
        if H.dtype != torch.float64 or not H.is_cuda:
            raise TypeError("H must be a float64 CUDA tensor")
        n = H.shape[0]
        if H1 is None:
            H1 = torch.empty(0, n, n, dtype=torch.float64, device=H.device)
        if H1.dtype != torch.float64 or not H1.is_cuda:
            raise TypeError("H1 must be a float64 CUDA tensor")
        if H1.dim() == 2:
            H1 = H1.unsqueeze(0)
        k = H1.shape[0]
        # a row-major view with a row stride ld >= n is passed as it is (the C
        # ABI's leading dimension); H1 must then hold its k blocks n * ld apart
        ld = H.stride(0)
        strided = (H.stride(1) == 1 and ld >= n and
                   (k == 0 or (H1.stride(2) == 1 and H1.stride(1) == ld and
                               H1.stride(0) == n * ld)))
        if not strided:
            H = H.contiguous()
            H1 = H1.contiguous()
            ld = n
        opts = options(precision=precision, **kw)
        if out is None:
            def alloc(*shape):   # outputs share the inputs' leading dimension
                full = torch.empty(*shape[:-1], ld, dtype=torch.float64, device=H.device)
                return full[..., :shape[-1]]
            P1 = alloc(k, n, n) if k else None
            P = alloc(n, n) if (want_P or k == 0) else None
        else:
            P, P1 = out
            for t, want in ((P, (ld, 1)), (P1, (n * ld, ld, 1))):
                if t is not None and tuple(t.stride()) != want:
                    raise ValueError("out tensors must have the inputs' leading dimension")
        nbytes = self.workspace_size(n, k, opts)
        if nbytes == 0:
            raise DmptError(1, "invalid sizes or options")
        if workspace is not None:
            if workspace.numel() < nbytes + 256:
                raise DmptError(2, "workspace tensor too small")
            ws_ptr = workspace.data_ptr() + ((-workspace.data_ptr()) % 256)
            ws_len = workspace.numel() - ((-workspace.data_ptr()) % 256)
        else:
            ws_ptr, ws_len = self.workspace(nbytes)
        info = DmptInfo()
        s = stream if stream is not None else torch.cuda.current_stream(H.device)
        st = self.lib.dmpt_sp2_response(
            self.h, H.data_ptr(), H1.data_ptr() if k else None, k, n, ld, int(n_occ),
            ctypes.byref(opts), P.data_ptr() if P is not None else None,
            P1.data_ptr() if P1 is not None else None, ctypes.byref(info),
            ctypes.c_void_p(ws_ptr), ws_len, ctypes.c_void_p(s.cuda_stream))
        inf = Info.from_c(info, k)
        if st != 0 and raise_on_error:
            self._check(st)
        return P, P1, inf

    def autotune(self, H, H1, n_occ: int, precision="dual_fp16", probe_layers=0, stream=None,
                 **kw):
        """Tune the layer-product configuration for (H, H1) (dmpt_autotune):
        returns (dict of the chosen cta_pair / tile_band / k_snake, ms per
        layer).  The handle keeps the result; calls with autotune=1 use it."""
        import torch
        if H1.dim() == 2:
            H1 = H1.unsqueeze(0)
        H, H1 = H.contiguous(), H1.contiguous()
        n, k = H.shape[0], H1.shape[0]
        opts = options(precision=precision, **kw)
        P = torch.empty(n, n, dtype=torch.float64, device=H.device)
        P1 = torch.empty(k, n, n, dtype=torch.float64, device=H.device) if k else None
        ws_ptr, ws_len = self.workspace(self.workspace_size(n, k, opts))
        best = DmptOptions()
        ms = ctypes.c_double(0.0)
        s = stream if stream is not None else torch.cuda.current_stream(H.device)
        st = self.lib.dmpt_autotune(self.h, H.data_ptr(), H1.data_ptr() if k else None, k, n, n,
                                    int(n_occ), ctypes.byref(opts), int(probe_layers), P.data_ptr(),
                                    P1.data_ptr() if k else None, ctypes.byref(best),
                                    ctypes.byref(ms), ctypes.c_void_p(ws_ptr), ws_len,
                                    ctypes.c_void_p(s.cuda_stream))
        self._check(st)
        return {"cta_pair": best.cta_pair, "tile_band": best.tile_band,
                "k_snake": best.k_snake}, ms.value

    def sp2_response2(self, H, H1, n_occ, precision="dual_fp16", stream=None,
                      raise_on_error=True, **kw):
        """P, P1 and the second-order response P2 = (1/2) d^2P/dlambda^2.
        Returns (P, P1 (k, n, n), P2 (k, n, n), Info); Info.d1_layer[k:] are
        the second-order stop layers."""
        import torch
        H = H.contiguous()
        if H1.dim() == 2:
            H1 = H1.unsqueeze(0)
        H1 = H1.contiguous()
        k, n = H1.shape[0], H.shape[0]
        opts = options(precision=precision, order=2, **kw)
        P = torch.empty_like(H)
        P1 = torch.empty_like(H1)
        P2 = torch.empty_like(H1)
        nbytes = self.workspace_size(n, k, opts)
        if nbytes == 0:
            raise DmptError(1, "invalid sizes or options")
        ws_ptr, ws_len = self.workspace(nbytes)
        info = DmptInfo()
        s = stream if stream is not None else torch.cuda.current_stream(H.device)
        st = self.lib.dmpt_sp2_response2(self.h, H.data_ptr(), H1.data_ptr(), k, n, n, int(n_occ),
                                         ctypes.byref(opts), P.data_ptr(), P1.data_ptr(),
                                         P2.data_ptr(), ctypes.byref(info), ctypes.c_void_p(ws_ptr),
                                         ws_len, ctypes.c_void_p(s.cuda_stream))
        if st != 0 and raise_on_error:
            self._check(st)
        return P, P1, P2, Info.from_c(info, 2 * k)

    def sp2_response_m(self, H, H1, n_occ, order, precision="dual_fp16", stream=None,
                       raise_on_error=True, **kw):
        """Responses of orders 1 .. order: P_o = (1/o!) d^o P / dlambda^o.
        Returns (P, [P_1, ..., P_order] each (k, n, n), Info); Info.d1_layer
        entries (o - 1) k .. o k - 1 are order o's stop layers."""
        import torch
        H = H.contiguous()
        if H1.dim() == 2:
            H1 = H1.unsqueeze(0)
        H1 = H1.contiguous()
        k, n = H1.shape[0], H.shape[0]
        opts = options(precision=precision, order=order, **kw)
        P = torch.empty_like(H)
        P1 = torch.empty_like(H1)
        Pk = torch.empty((max(order - 1, 0) * k, n, n), dtype=H.dtype, device=H.device)
        nbytes = self.workspace_size(n, k, opts)
        if nbytes == 0:
            raise DmptError(1, "invalid sizes or options")
        ws_ptr, ws_len = self.workspace(nbytes)
        info = DmptInfo()
        s = stream if stream is not None else torch.cuda.current_stream(H.device)
        st = self.lib.dmpt_sp2_response_m(self.h, H.data_ptr(), H1.data_ptr(), k, n, n,
                                          int(n_occ), int(order), ctypes.byref(opts),
                                          P.data_ptr(), P1.data_ptr(),
                                          Pk.data_ptr() if order >= 2 else None,
                                          ctypes.byref(info), ctypes.c_void_p(ws_ptr), ws_len,
                                          ctypes.c_void_p(s.cuda_stream))
        if st != 0 and raise_on_error:
            self._check(st)
        terms = [P1] + [Pk[(o - 2) * k:(o - 1) * k] for o in range(2, order + 1)]
        return P, terms, Info.from_c(info, order * k)

    def sp2_backward(self, G, workspace, out=None, stream=None, **kw):
        """dL/dH of L = Tr[G P] for the forward run that filled `workspace`
        (a uint8 CUDA tensor used with ckpt_every >= 1: the full S0 tape, or
        checkpoints every ckpt_every states with recomputation)."""
        import torch
        if G.dtype != torch.float64 or not G.is_cuda:
            raise TypeError("G must be a float64 CUDA tensor")
        G = G.contiguous()
        n = G.shape[0]
        dLdH = torch.empty_like(G) if out is None else out
        opts = options(**kw)
        ws_ptr = workspace.data_ptr() + ((-workspace.data_ptr()) % 256)
        ws_len = workspace.numel() - ((-workspace.data_ptr()) % 256)
        s = stream if stream is not None else torch.cuda.current_stream(G.device)
        self._check(self.lib.dmpt_sp2_backward(self.h, G.data_ptr(), n, n, ctypes.byref(opts),
                                               dLdH.data_ptr(), ctypes.c_void_p(ws_ptr), ws_len,
                                               ctypes.c_void_p(s.cuda_stream)))
        return dLdH

    def sp2_response_batch(self, Hs, H1s, n_occs, precision="dual_fp16", stream=None,
                           raise_on_error=True, **kw):
        """Independent instances (lists of float64 CUDA tensors) in one call.
        Returns (list of P, list of P1 (k, n, n) or None, list of Info)."""
        import torch
        count = len(Hs)
        Hs = [h.contiguous() for h in Hs]
        k = 0 if H1s is None else (H1s[0].shape[0] if H1s[0].dim() == 3 else 1)
        if H1s is not None:
            H1s = [(h1 if h1.dim() == 3 else h1.unsqueeze(0)).contiguous() for h1 in H1s]
        ns = [h.shape[0] for h in Hs]
        Ps = [torch.empty_like(h) for h in Hs]
        P1s = [torch.empty(k, n, n, dtype=torch.float64, device=h.device) for n, h in zip(ns, Hs)] if k else None
        opts = options(precision=precision, **kw)
        I64 = ctypes.c_int64 * count
        VP = ctypes.c_void_p * count
        n_arr = I64(*ns)
        nbytes = self.lib.dmpt_workspace_size_batch(count, n_arr, k, ctypes.byref(opts))
        if nbytes == 0:
            raise DmptError(1, "invalid batch sizes or options")
        ws_ptr, ws_len = self.workspace(nbytes)
        infos = (DmptInfo * count)()
        s = stream if stream is not None else torch.cuda.current_stream(Hs[0].device)
        st = self.lib.dmpt_sp2_response_batch(
            self.h, count, VP(*[h.data_ptr() for h in Hs]),
            VP(*[h1.data_ptr() for h1 in H1s]) if k else None, k, n_arr, I64(*ns),
            I64(*[int(x) for x in n_occs]), ctypes.byref(opts), VP(*[p.data_ptr() for p in Ps]),
            VP(*[p.data_ptr() for p in P1s]) if k else None, infos, ctypes.c_void_p(ws_ptr),
            ws_len, ctypes.c_void_p(s.cuda_stream))
        if st != 0 and raise_on_error:
            self._check(st)
        return Ps, P1s, [Info.from_c(infos[i], k) for i in range(count)]

    @staticmethod
    def _ws_ptr(workspace):
        off = (-workspace.data_ptr()) % 256
        return workspace.data_ptr() + off, workspace.numel() - off

    def response_replay(self, H1, workspace, out=None, stream=None, **kw):
        """P1 for new perturbations H1 ((n, n) or (k, n, n)) from the S0 tape
        of the forward run that filled `workspace` (ckpt_every=1)."""
        import torch
        if H1.dim() == 2:
            H1 = H1.unsqueeze(0)
        H1 = H1.contiguous()
        k, n = H1.shape[0], H1.shape[1]
        P1 = torch.empty_like(H1) if out is None else out
        opts = options(**kw)
        info = DmptInfo()
        ptr, ln = self._ws_ptr(workspace)
        s = stream if stream is not None else torch.cuda.current_stream(H1.device)
        self._check(self.lib.dmpt_response_replay(self.h, H1.data_ptr(), k, n, n,
                                                  ctypes.byref(opts), P1.data_ptr(),
                                                  ctypes.byref(info), ctypes.c_void_p(ptr), ln,
                                                  ctypes.c_void_p(s.cuda_stream)))
        return P1, Info.from_c(info, k)

    def scc_response(self, H1_ext, gamma, workspace, tol=1e-6, max_iter=100, mixing=0.8,
                     out=None, stream=None, raise_on_error=True, **kw):
        """Self-consistent P1 (H1 = H1_ext + diag(gamma diag(P1))) from the S0
        tape of the forward run that filled `workspace`.  Returns
        (P1, iterations, residual, Info)."""
        import torch
        if H1_ext.dim() == 2:
            H1_ext = H1_ext.unsqueeze(0)
        H1_ext = H1_ext.contiguous()
        gamma = gamma.contiguous()
        k, n = H1_ext.shape[0], H1_ext.shape[1]
        P1 = torch.empty_like(H1_ext) if out is None else out
        opts = options(**kw)
        info = DmptInfo()
        its = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        ptr, ln = self._ws_ptr(workspace)
        s = stream if stream is not None else torch.cuda.current_stream(H1_ext.device)
        st = self.lib.dmpt_scc_response(self.h, H1_ext.data_ptr(), gamma.data_ptr(), k, n, n,
                                        ctypes.byref(opts), float(tol), int(max_iter),
                                        float(mixing), P1.data_ptr(), ctypes.byref(info),
                                        ctypes.byref(its), ctypes.byref(res),
                                        ctypes.c_void_p(ptr), ln, ctypes.c_void_p(s.cuda_stream))
        if st != 0 and raise_on_error:
            self._check(st)
        return P1, its.value, res.value, Info.from_c(info, k)

    def host_copy_in_bytes(self, n: int, k: int) -> int:
        """Bytes solve_host copies to the device per instance (the upper
        triangles of H and the k perturbations)."""
        return int(self.lib.dmpt_host_copy_in_bytes(n, k))

    def solve_host(self, Hs, H1s, n_occ: int, P1_out=None, P_out=None, precision="dual_fp16",
                   stream=None, raise_on_error=True, workspace=None, **kw):
        """Instances held in host memory (dmpt_sp2_response_host): lists of
        (n, n) and (k, n, n) float64 CPU tensors, pinned for the copies to
        overlap the solves; only their upper triangles are read.  Results go to `P1_out` / `P_out` (lists of CPU
        tensors, allocated pinned when None; P is copied out only when
        `P_out` is given).  Returns (P list or None, P1 list, Info list)."""
        import torch
        count = len(Hs)
        n = Hs[0].shape[0]
        Hs = [h if h.is_contiguous() else h.contiguous() for h in Hs]
        H1s = [(h1 if h1.dim() == 3 else h1.unsqueeze(0)) for h1 in H1s]
        H1s = [h1 if h1.is_contiguous() else h1.contiguous() for h1 in H1s]
        k = H1s[0].shape[0]
        for h, h1 in zip(Hs, H1s):
            if h.device.type != "cpu" or h1.device.type != "cpu" or h.dtype != torch.float64 \
                    or h1.dtype != torch.float64 or h.shape != (n, n) or h1.shape != (k, n, n):
                raise ValueError("solve_host wants float64 CPU tensors of one size")
        if P1_out is None:
            P1_out = [torch.empty(k, n, n, dtype=torch.float64).pin_memory() for _ in range(count)]
        opts = options(precision=precision, **kw)
        nbytes = self.lib.dmpt_workspace_size_host(n, k, ctypes.byref(opts))
        if nbytes == 0:
            raise DmptError(1, "invalid size or options")
        if workspace is not None:
            if workspace.numel() < nbytes + 256:
                raise DmptError(2, "workspace tensor too small")
            ws_ptr, ws_len = self._ws_ptr(workspace)
        else:
            ws_ptr, ws_len = self.workspace(nbytes)
        dev = torch.device(f"cuda:{self.device}")
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        VP = ctypes.c_void_p * count
        infos = (DmptInfo * count)()
        st = self.lib.dmpt_sp2_response_host(
            self.h, count, VP(*[h.data_ptr() for h in Hs]), VP(*[h1.data_ptr() for h1 in H1s]), k,
            n, int(n_occ), ctypes.byref(opts),
            VP(*[p.data_ptr() for p in P_out]) if P_out is not None else None,
            VP(*[p.data_ptr() for p in P1_out]), infos, ctypes.c_void_p(ws_ptr), ws_len,
            ctypes.c_void_p(s.cuda_stream))
        if st != 0 and raise_on_error:
            self._check(st)
        return P_out, P1_out, [Info.from_c(infos[i], k) for i in range(count)]

    def sp2_response_host(self, H_host, H1_host, n_occ: int, precision="dual_fp16",
                          stream=None, **kw):
        """One instance from host (CPU, ideally pinned) tensors through the C
        ABI's host entry point: copy in, solve, copy out.  Returns (P, P1, Info)."""
        import torch
        n = H_host.shape[0]
        P = torch.empty(n, n, dtype=torch.float64).pin_memory()
        Ps, P1s, infos = self.solve_host([H_host], [H1_host], n_occ, P_out=[P],
                                         precision=precision, stream=stream, **kw)
        return Ps[0], P1s[0], infos[0]


_default_ctx: Optional[Context] = None


def context(device: int = 0) -> Context:
    global _default_ctx
    if _default_ctx is None or _default_ctx.device != device:
        _default_ctx = Context(device)
    return _default_ctx


def sp2_response(H, H1, n_occ, precision="dual_fp16", **kw):
    """Module-level convenience wrapper around Context.sp2_response."""
    return context(H.device.index or 0).sp2_response(H, H1, n_occ, precision=precision, **kw)


def bounds(H):
    return context(H.device.index or 0).bounds(H)


def _autograd_function():
    import torch

    class SP2Density(torch.autograd.Function):
        """P = theta(mu I - H) by DNN-SP2-PT with the hand-written adjoint.

        forward(H, n_occ, precision, ckpt_every): runs dmpt_sp2_response with
        k = 0 and the S0 states (every state for ckpt_every = 1, else an FP32
        checkpoint of every ckpt_every-th state) kept in a workspace owned by
        this node; backward(gP) runs dmpt_sp2_backward on it.
        """

        @staticmethod
        def forward(ctx, H, n_occ, precision="dual_fp16", ckpt_every=8):
            c = context(H.device.index or 0)
            opts = options(precision=precision, ckpt_every=ckpt_every)
            nbytes = c.workspace_size(H.shape[0], 0, opts)
            ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=H.device)
            P, _, info = c.sp2_response(H.detach(), None, n_occ, precision=precision,
                                        ckpt_every=ckpt_every, workspace=ws)
            ctx.ws = ws
            ctx.info = info
            return P

        @staticmethod
        def backward(ctx, gP):
            c = context(gP.device.index or 0)
            dLdH = c.sp2_backward(gP.detach().to(torch.float64), ctx.ws)
            return dLdH, None, None, None

    return SP2Density


_sp2_density = None


def density(H, n_occ, precision="dual_fp16", ckpt_every=8):
    """Differentiable P(H): torch.autograd-aware wrapper of the CUDA path.

    ckpt_every: 1 keeps every S0 state for the backward; k >= 2 keeps an FP32
    checkpoint of every k-th state and recomputes the rest (default 8)."""
    global _sp2_density
    if _sp2_density is None:
        _sp2_density = _autograd_function()
    return _sp2_density.apply(H, n_occ, precision, ckpt_every)

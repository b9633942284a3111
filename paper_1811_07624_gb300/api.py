"""Python face of libhh: a plan object over torch CUDA tensors.

The calls pass tensor pointers, leading dimensions and the current torch
stream to the C ABI (``include/hh.h``); PyTorch only provides device memory
and streams.  Transform (§II-A Eq. (1), §III-A Eq. (21)): W = H_1 ... H_h,
H_k = I - 2 u_k u_k^T, u_k = v_k / |v_k|;

    apply(X)      -> sigma .* (W x)                        per row x of X
    apply_T(X)    -> W^T (sigma .* x)
    apply_sym(X)  -> sigma .* W (d .* W^T (sigma .* x))
"""

from __future__ import annotations

import ctypes

import torch

from . import _lib

_TORCH_DTYPES = {torch.float32: "f32", torch.float64: "f64", torch.bfloat16: "bf16"}


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _rows(t: torch.Tensor, name: str, n: int, dtype: torch.dtype):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} has dtype {t.dtype}, the plan computes in {dtype}")
    if t.dim() != 2 or t.shape[1] != n:
        raise ValueError(f"{name} must have shape (batch, {n}), got {tuple(t.shape)}")
    if t.shape[0] > 0 and t.stride(1) != 1:
        raise ValueError(f"{name} rows must be contiguous (stride(1) == 1)")
    ld = t.stride(0) if t.shape[0] > 1 else max(t.stride(0), n)
    return t.data_ptr(), max(ld, n)


class Plan:
    """A created transform: h reflectors of length n, optional spectrum and sign.

    U: CUDA tensor (h, n) of float32, float64 or bfloat16 (rows are v_k, any
    non-zero norm; zero rows are identity factors).  d: optional (n,) spectrum.
    sign: optional (n,) tensor of +-1 (converted to int8).  path: "auto",
    "fused" or "wy".
    """

    def __init__(self, U: torch.Tensor, d: torch.Tensor | None = None,
                 sign: torch.Tensor | None = None, path: str = "auto", stream=None):
        if U.dim() != 2:
            raise ValueError("U must be 2-D (h, n)")
        if U.dtype not in _TORCH_DTYPES:
            raise ValueError(f"unsupported dtype {U.dtype}")
        if not U.is_cuda:
            raise ValueError("U must be a CUDA tensor")
        self.h, self.n = int(U.shape[0]), int(U.shape[1])
        self.dtype = U.dtype
        U = U.contiguous()
        dd = None
        if d is not None:
            dd = d.to(device=U.device, dtype=U.dtype).contiguous()
            if dd.shape != (self.n,):
                raise ValueError("d must have shape (n,)")
        ss = None
        if sign is not None:
            ss = sign.to(device=U.device, dtype=torch.int8).contiguous()
            if ss.shape != (self.n,):
                raise ValueError("sign must have shape (n,)")
        self.has_d = dd is not None
        self.device = U.device
        handle = ctypes.c_void_p()
        with torch.cuda.device(U.device):
            _lib.call("hh_create_ex", ctypes.byref(handle), self.n, self.h,
                      U.data_ptr() if self.h > 0 else None, self.n,
                      dd.data_ptr() if dd is not None else None,
                      ss.data_ptr() if ss is not None else None,
                      _lib.DTYPES[_TORCH_DTYPES[U.dtype]], _lib.PATHS[path],
                      _stream_ptr(stream))
        self._h = handle
        # incremented by update(): an autograd graph built before an update
        # must not run its backward with the new reflector values
        self.generation = 0
        n64, h64, dt, pa = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        _lib.call("hh_plan_info", self._h, ctypes.byref(n64), ctypes.byref(h64),
                  ctypes.byref(dt), ctypes.byref(pa))
        self.path = {v: k for k, v in _lib.PATHS.items()}[pa.value]

    # -- lifetime ---------------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.call("hh_destroy", self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sync(self, stream=None) -> None:
        """Wait for this plan's work on the stream; raise if a kernel timed out."""
        _lib.call("hh_sync", self._h, _stream_ptr(stream))

    def update(self, U: torch.Tensor, d: torch.Tensor | None = None, stream=None) -> None:
        """New reflector rows (and spectrum, if the plan has one) for this F32/F64
        plan, stream-ordered, without allocation or host synchronisation."""
        if U.shape != (self.h, self.n) or U.dtype != self.dtype or not U.is_cuda:
            raise ValueError(f"U must be a CUDA {self.dtype} tensor of shape ({self.h}, {self.n})")
        if self.h and U.stride(1) != 1:
            raise ValueError("U rows must be contiguous")
        ldu = U.stride(0) if self.h > 1 else self.n
        dp = None
        if d is not None:
            if d.shape != (self.n,) or d.dtype != self.dtype or not d.is_cuda or d.stride(0) != 1:
                raise ValueError(f"d must be a contiguous CUDA {self.dtype} tensor of shape ({self.n},)")
            dp = d.data_ptr()
        _lib.call("hh_update", self._h, U.data_ptr() if self.h else None, max(ldu, self.n), dp,
                  _stream_ptr(stream))
        self.generation += 1

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def skip_prefix(self, mode: int | None = None) -> bool:
        """Skipping of the reflectors' zero prefixes (§II-D): True/1 on, False/0
        off, -1 back to the automatic choice made at create; None only reads.
        Returns the setting in force."""
        out = ctypes.c_int()
        _lib.call("hh_plan_skip_prefix", self._h, -2 if mode is None else int(mode),
                  ctypes.byref(out))
        return bool(out.value)

    # -- forward ------------------------------------------------------------------
    def _apply(self, fn: str, X: torch.Tensor, out: torch.Tensor | None, stream) -> torch.Tensor:
        xp, ldx = _rows(X, "X", self.n, self.dtype)
        if out is None:
            out = torch.empty((X.shape[0], self.n), device=X.device, dtype=self.dtype)
        yp, ldy = _rows(out, "out", self.n, self.dtype)
        if out.shape[0] != X.shape[0]:
            raise ValueError("out must have as many rows as X")
        _lib.call(fn, self._h, xp, ldx, yp, ldy, X.shape[0], _stream_ptr(stream))
        return out

    def apply(self, X, out=None, stream=None):
        """sigma .* (W x) per row (Eq. (1))."""
        return self._apply("hh_apply", X, out, stream)

    def apply_T(self, X, out=None, stream=None):
        """W^T (sigma .* x) per row."""
        return self._apply("hh_apply_T", X, out, stream)

    def apply_sym(self, X, out=None, stream=None):
        """sigma .* W (d .* W^T (sigma .* x)) per row (Eq. (21))."""
        return self._apply("hh_apply_sym", X, out, stream)

    def apply_sym_p(self, X, out=None, p_out=None, stream=None):
        """apply_sym that also returns p = W^T (sigma .* x), the state between the
        halves of Eq. (21), for ``backward("SYM", None, gY, Y=y, P=p)``.  Returns (y, p)."""
        xp, ldx = _rows(X, "X", self.n, self.dtype)
        B = X.shape[0]
        if out is None:
            out = torch.empty((B, self.n), device=X.device, dtype=self.dtype)
        if p_out is None:
            p_out = torch.empty((B, self.n), device=X.device, dtype=self.dtype)
        yp, ldy = _rows(out, "out", self.n, self.dtype)
        pp, ldp = _rows(p_out, "p_out", self.n, self.dtype)
        if out.shape[0] != B or p_out.shape[0] != B:
            raise ValueError("out and p_out must have as many rows as X")
        _lib.call("hh_apply_sym_p", self._h, xp, ldx, yp, ldy, pp, ldp, B, _stream_ptr(stream))
        return out, p_out

    def apply_mode(self, mode: str, X, out=None, stream=None):
        return {"W": self.apply, "WT": self.apply_T, "SYM": self.apply_sym}[mode](X, out, stream)

    # -- backward -----------------------------------------------------------------
    def backward(self, mode: str, saved, gY, need_gX: bool = True, need_gU: bool = True,
                 need_gd: bool | None = None, stream=None, Y=None, P=None):
        """Gradients of L with dL/dY = gY through ``apply_mode(mode, X)``.

        saved: the forward output Y for modes "W" and "WT", the forward input X
        for "SYM".  For "SYM", Y may give the forward output as well
        (``apply_sym(X)`` of this plan): the adjoint then reads its state from
        it instead of recomputing it (hh_backward_sym_y); with Y and P from
        ``apply_sym_p(X)``, saved may be None (hh_backward_sym_py).  Returns
        (gX, gU, gd); gU (h, n) is the gradient with respect to the reflector
        rows exactly as passed to the plan; gd (n,) only for SYM.
        """
        m = _lib.MODES[mode]
        if mode == "SYM" and P is not None:
            if Y is None:
                raise ValueError("P needs Y as well")
            saved = P
        sp, lds = _rows(saved, "saved", self.n, self.dtype)
        gp, ldg = _rows(gY, "gY", self.n, self.dtype)
        if saved.shape[0] != gY.shape[0]:
            raise ValueError("saved and gY must have the same number of rows")
        B = saved.shape[0]
        dev = saved.device
        gX = torch.empty((B, self.n), device=dev, dtype=self.dtype) if need_gX else None
        gU = torch.empty((self.h, self.n), device=dev, dtype=self.dtype) if need_gU and self.h else None
        if need_gd is None:
            need_gd = mode == "SYM"
        gd = torch.empty((self.n,), device=dev, dtype=self.dtype) if need_gd and mode == "SYM" else None
        xp, ldgx = (None, self.n) if gX is None else _rows(gX, "gX", self.n, self.dtype)
        up = None if gU is None else gU.data_ptr()
        dp = None if gd is None else gd.data_ptr()
        if Y is not None and mode == "SYM":
            yp, ldy = _rows(Y, "Y", self.n, self.dtype)
            if Y.shape[0] != B:
                raise ValueError("Y and saved must have the same number of rows")
            fn = "hh_backward_sym_py" if P is not None else "hh_backward_sym_y"
            _lib.call(fn, self._h, sp, lds, yp, ldy, gp, ldg, xp, ldgx, up, dp, B,
                      _stream_ptr(stream))
        else:
            _lib.call("hh_backward", self._h, m, sp, lds, gp, ldg, xp, ldgx, up, dp, B,
                      _stream_ptr(stream))
        if need_gU and self.h == 0:
            gU = torch.zeros((0, self.n), device=dev, dtype=self.dtype)
        return gX, gU, gd

    # -- fast Mahalanobis distance (§IV-C) ------------------------------------------
    def mahalanobis(self, X, ia, ib, out=None, stream=None):
        """d_S(x_ia[p], x_ib[p]) = sum_m d_m [W^T(sigma.*(x_a - x_b))]_m^2 for each pair."""
        xp, ldx = _rows(X, "X", self.n, self.dtype)
        ia = ia.to(device=X.device, dtype=torch.int64).contiguous()
        ib = ib.to(device=X.device, dtype=torch.int64).contiguous()
        if ia.shape != ib.shape or ia.dim() != 1:
            raise ValueError("ia, ib must be equal-length 1-D index tensors")
        P = ia.shape[0]
        if out is None:
            out = torch.empty((P,), device=X.device, dtype=self.dtype)
        _lib.call("hh_mahalanobis", self._h, xp, ldx, X.shape[0], ia.data_ptr(), ib.data_ptr(),
                  P, out.data_ptr(), _stream_ptr(stream))
        return out

    def mahalanobis_backward(self, X, ia, ib, gout, need_gU=True, need_gd=True, stream=None):
        """(gU, gd) of L = sum_p gout[p] d_S(x_ia[p], x_ib[p])."""
        xp, ldx = _rows(X, "X", self.n, self.dtype)
        ia = ia.to(device=X.device, dtype=torch.int64).contiguous()
        ib = ib.to(device=X.device, dtype=torch.int64).contiguous()
        gout = gout.to(device=X.device, dtype=self.dtype).contiguous()
        gU = torch.empty((self.h, self.n), device=X.device, dtype=self.dtype) if need_gU and self.h else None
        gd = torch.empty((self.n,), device=X.device, dtype=self.dtype) if need_gd else None
        _lib.call("hh_mahalanobis_backward", self._h, xp, ldx, X.shape[0], ia.data_ptr(),
                  ib.data_ptr(), ia.shape[0], gout.data_ptr(),
                  None if gU is None else gU.data_ptr(), None if gd is None else gd.data_ptr(),
                  _stream_ptr(stream))
        if need_gU and self.h == 0:
            gU = torch.zeros((0, self.n), device=X.device, dtype=self.dtype)
        return gU, gd


# -- batched persistent launch ------------------------------------------------------
class Batch:
    """Many transforms applied in one graph-replayed launch (hh_batch_*).

    plans: F32 plans (n % 4 == 0, n <= 4096); batches: rows per plan.  The
    tile shape of each transform comes from the autotuner's table at creation
    (:func:`tune`, :func:`tune_load`, :func:`tune_set`): a staged shape, run by
    one persistent kernel on a shared work counter, or the resident-reflector
    shape (n <= 2048, h <= 100), run by one kernel per cluster size on a static
    schedule; all of them replay as one CUDA graph.  The batch keeps its plans
    alive.
    """

    def __init__(self, plans, batches):
        self.plans = list(plans)
        self.batches = [int(b) for b in batches]
        if len(self.plans) != len(self.batches):
            raise ValueError("plans and batches differ in length")
        for p in self.plans:
            if p.dtype != torch.float32:
                raise ValueError("the batched launch takes float32 plans only")
        count = len(self.plans)
        hs = (ctypes.c_void_p * max(count, 1))(*[p.handle.value for p in self.plans])
        bs = (ctypes.c_int64 * max(count, 1))(*self.batches)
        self._h = ctypes.c_void_p()
        _lib.call("hh_batch_create", ctypes.byref(self._h), count, hs, bs)

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.call("hh_batch_destroy", self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def apply(self, Xs, Ys=None, mode: str = "W", stream=None):
        """Ys[i] = op(Xs[i]) for every transform, op = W, WT or SYM; one launch."""
        count = len(self.plans)
        if len(Xs) != count:
            raise ValueError(f"expected {count} inputs, got {len(Xs)}")
        if Ys is None:
            Ys = [torch.empty_like(X) for X in Xs]
        if len(Ys) != count:
            raise ValueError(f"expected {count} outputs, got {len(Ys)}")
        # the marshalled pointer arrays are kept while the tensors' pointers,
        # shapes and strides stay the same (the usual case: one set of buffers)
        key = tuple((X.data_ptr(), tuple(X.shape), X.stride(), X.dtype, X.device,
                     Y.data_ptr(), tuple(Y.shape), Y.stride(), Y.dtype, Y.device)
                    for X, Y in zip(Xs, Ys))
        cache = getattr(self, "_marshalled", None)
        if cache is None or cache[0] != key:
            xp, yp, lx, ly = [], [], [], []
            for i, (p, X, Y, b) in enumerate(zip(self.plans, Xs, Ys, self.batches)):
                if X.shape[0] != b or Y.shape[0] != b:
                    raise ValueError(f"transform {i}: expected {b} rows")
                a, la = _rows(X, f"Xs[{i}]", p.n, torch.float32)
                c, lc = _rows(Y, f"Ys[{i}]", p.n, torch.float32)
                xp.append(a)
                yp.append(c)
                lx.append(la)
                ly.append(lc)
            n = max(count, 1)
            cache = (key, (ctypes.c_void_p * n)(*xp), (ctypes.c_int64 * n)(*lx),
                     (ctypes.c_void_p * n)(*yp), (ctypes.c_int64 * n)(*ly))
            self._marshalled = cache
        _lib.call("hh_batch_apply", self._h, _lib.MODES[mode], cache[1], cache[2], cache[3],
                  cache[4], _stream_ptr(stream))
        return Ys

    def sync(self, stream=None) -> None:
        _lib.call("hh_batch_sync", self._h, _stream_ptr(stream))

    def info(self) -> dict:
        count = len(self.plans)
        ni = ctypes.c_int64()
        grid = ctypes.c_int()
        shapes = (ctypes.c_int * max(count, 1))()
        _lib.call("hh_batch_info", self._h, ctypes.byref(ni), ctypes.byref(grid), shapes)
        return {"items": ni.value, "grid": grid.value, "shapes": list(shapes)[:count]}


def batch_shapes() -> list[dict]:
    """The tile shapes compiled into the batched kernel: G, NG, RT, rows_per_tile,
    cover, max_h (-1: no limit) and max_cluster (CTAs per cluster of the
    resident-reflector shape; 0 for a staged shape)."""
    out = []
    for s in range(_lib.lib().hh_batch_num_shapes()):
        v = [ctypes.c_int() for _ in range(5)]
        _lib.call("hh_batch_shape", s, *[ctypes.byref(x) for x in v])
        d = dict(zip(("G", "NG", "RT", "rows_per_tile", "cover"), [x.value for x in v]))
        mh, mc = ctypes.c_int(), ctypes.c_int()
        _lib.call("hh_batch_shape_limits", s, ctypes.byref(mh), ctypes.byref(mc))
        d.update(max_h=mh.value, max_cluster=mc.value)
        out.append(d)
    return out


def tune(ns, hs, rows: int = 16384, stream=None) -> None:
    """Time every tile shape for each (n, h) and keep the fastest (hh_tune)."""
    ns, hs = [int(n) for n in ns], [int(h) for h in hs]
    _lib.call("hh_tune", (ctypes.c_int64 * max(len(ns), 1))(*ns), len(ns),
              (ctypes.c_int64 * max(len(hs), 1))(*hs), len(hs), int(rows), _stream_ptr(stream))


def tune_get(n: int, h: int):
    """(shape the batch would use for (n, h), measured ms per shape or NaN)."""
    shape = ctypes.c_int()
    ms = (ctypes.c_float * _lib.lib().hh_batch_num_shapes())()
    _lib.call("hh_tune_get", int(n), int(h), ctypes.byref(shape), ms)
    return shape.value, list(ms)


def tune_set(n: int, h: int, shape: int) -> None:
    _lib.call("hh_tune_set", int(n), int(h), int(shape))


def tune_save(path: str) -> None:
    _lib.call("hh_tune_save", str(path).encode())


def tune_load(path: str) -> None:
    _lib.call("hh_tune_load", str(path).encode())


def tune_clear() -> None:
    _lib.call("hh_tune_clear")

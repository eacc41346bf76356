"""PyTorch front end: device memory and streams come from torch, all compute
from liblegcheb.so (see binding.py).  No CPU path exists."""
from __future__ import annotations

import torch

from . import binding as B

_DIRECTIONS = {"l2c": B.LC_L2C, "c2l": B.LC_C2L}
_DTYPES = {"f64": B.LC_F64, "f64_split": B.LC_F64_SPLIT, "f32": B.LC_F32, "f64_df": B.LC_F64_DF}
_TORCH_DTYPE = {B.LC_F64: torch.float64, B.LC_F64_SPLIT: torch.float64, B.LC_F32: torch.float32,
                B.LC_F64_DF: torch.float64}


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def make_options(s_hat: int | None = None, fixed_s: int | None = None, slices: int | None = None,
                 debug_flags: int | None = None, values: bool | None = None, alpha: float | None = None,
                 nodal: bool | None = None, fp64_plan: bool | None = None):
    o = B.lc_plan_options_default()
    if fp64_plan is not None:
        o.fp64_plan = int(bool(fp64_plan))
    if nodal is not None:
        o.nodal = int(bool(nodal))
    if alpha is not None:
        o.alpha = float(alpha)
    if values is not None:
        o.values = int(bool(values))
    if debug_flags is not None:
        o.debug_flags = debug_flags
    if s_hat is not None:
        o.s_hat = s_hat
    if fixed_s is not None:
        o.fixed_s = fixed_s
    if slices is not None:
        o.slices = slices
    return o


class Plan:
    """A transform plan: tables built on the GPU in a torch-owned workspace.

    direction: "l2c" (f_cheb = C^{-1} A f_leg) or "c2l" (f_leg = A^{-1} C f_cheb)
    dtype:     "f64" | "f64_split" | "f32" | "f64_df"
    lengths:   for a ragged plan, the member lengths (then n and batch are ignored)
    values:    True: the Chebyshev side holds values at the n Chebyshev-Gauss points
               cos((m + 1/2) pi / n) instead of coefficients ("l2c": Legendre synthesis
               on those points; "c2l": Legendre coefficients from the values)
    alpha:     Gegenbauer parameter a (-1/2 < a <= 2, a != 0): the non-Chebyshev side
               holds coefficients of C_j^(a) instead of P_j = C_j^(1/2) (default: Legendre)
    nodal:     True: the nodal (Lagrange) variant of the far field instead of the modal
               one ("f64" and "f32" only); the same map
    """

    def __init__(self, n: int | None = None, direction: str = "l2c", batch: int = 1, dtype: str = "f64",
                 device=None, lengths=None, **options):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.direction = _DIRECTIONS[direction]
        self.dtype_code = _DTYPES[dtype]
        self.dtype_name = dtype
        self.torch_dtype = _TORCH_DTYPE[self.dtype_code]
        self.options = make_options(**options)
        self._handle = None
        with torch.cuda.device(self.device):
            st = _stream_ptr(self.device)
            if lengths is not None:
                self.lengths = [int(v) for v in lengths]
                self.ragged = True
                nbytes = B.lc_plan_workspace_size_ragged(self.lengths, self.direction, self.dtype_code, self.options)
                self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
                self._handle = B.lc_plan_create_ragged(self.lengths, self.direction, self.dtype_code,
                                                       self.workspace.data_ptr(), nbytes, st, self.options)
                self.total = sum(self.lengths)
            else:
                self.ragged = False
                nbytes = B.lc_plan_workspace_size(n, self.direction, batch, self.dtype_code, self.options)
                self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
                self._handle = B.lc_plan_create(n, self.direction, batch, self.dtype_code,
                                                self.workspace.data_ptr(), nbytes, st, self.options)
        self.info = B.lc_plan_info(self._handle)
        self.n = self.info["n"]
        self.batch = self.info["batch"]

    # ------------------------------------------------------------------ run
    def _check_in(self, x: torch.Tensor):
        if x.device != self.device or x.dtype != self.torch_dtype:
            raise TypeError("expected a %s tensor on %s, got %s on %s" % (self.torch_dtype, self.device, x.dtype, x.device))

    def _strides(self, x: torch.Tensor):
        if self.ragged:
            if x.dim() != 1 or x.numel() != self.total or x.stride(0) != 1:
                raise ValueError("ragged input must be a contiguous 1-D tensor of %d elements" % self.total)
            return 0, 1
        if x.dim() == 1:
            if self.batch != 1 or x.shape[0] != self.n:
                raise ValueError("expected shape (%d,)" % self.n)
            return 0, x.stride(0)
        if x.dim() != 2 or tuple(x.shape) != (self.batch, self.n):
            raise ValueError("expected shape (%d, %d)" % (self.batch, self.n))
        return x.stride(0), x.stride(1)

    def __call__(self, x: torch.Tensor, out: torch.Tensor | None = None, adjoint: bool = False) -> torch.Tensor:
        return self.execute(x, out=out, adjoint=adjoint)

    def execute(self, x: torch.Tensor, out: torch.Tensor | None = None, adjoint: bool = False) -> torch.Tensor:
        self._check_in(x)
        ib, ie = self._strides(x)
        if out is None:
            out = torch.empty_like(x, memory_format=torch.contiguous_format) if x.dim() > 0 else torch.empty_like(x)
        else:
            self._check_in(out)
        ob, oe = self._strides(out)
        fn = B.lc_adjoint if adjoint else B.lc_execute
        with torch.cuda.device(self.device):
            fn(self._handle, x.data_ptr(), out.data_ptr(), ib, ie, ob, oe, _stream_ptr(self.device))
        return out

    def execute_strided(self, x: torch.Tensor, out: torch.Tensor, in_strides, out_strides, adjoint: bool = False):
        """Raw strided call: vector b, element j at x.data_ptr() + (b*sb + j*se) elements."""
        self._check_in(x)
        self._check_in(out)
        fn = B.lc_adjoint if adjoint else B.lc_execute
        with torch.cuda.device(self.device):
            fn(self._handle, x.data_ptr(), out.data_ptr(), in_strides[0], in_strides[1], out_strides[0],
               out_strides[1], _stream_ptr(self.device))
        return out

    def execute_strided2(self, x: torch.Tensor, out: torch.Tensor, in_strides, out_strides, batch_inner: int,
                         adjoint: bool = False):
        """Two-level strided call (lc_execute_ex): vector b, element j at
        x.data_ptr() + ((b // batch_inner) * so + (b % batch_inner) * sb + j * se)
        elements, with in_strides = (sb, se, so) and out_strides likewise."""
        self._check_in(x)
        self._check_in(out)
        fn = B.lc_adjoint_ex if adjoint else B.lc_execute_ex
        with torch.cuda.device(self.device):
            fn(self._handle, x.data_ptr(), out.data_ptr(), in_strides[0], in_strides[1], out_strides[0],
               out_strides[1], batch_inner, in_strides[2], out_strides[2], _stream_ptr(self.device))
        return out

    def along_axis(self, x: torch.Tensor, axis: int, out: torch.Tensor | None = None, adjoint: bool = False):
        """Transform every fibre of a contiguous 3-D array along `axis` (0, 1 or 2)
        in one call, writing the result in the same layout (a new array unless
        `out` is given).  The plan's n must equal x.shape[axis] and its batch the
        product of the other two extents."""
        if x.dim() != 3 or not x.is_contiguous():
            raise ValueError("expected a contiguous 3-D tensor")
        P, Nn, Q = x.shape
        if out is None:
            out = torch.empty_like(x)
        if axis == 0:    # fibre (j, k): batch index j*Q + k (stride 1), element stride Nn*Q
            self.execute_strided(x, out, (1, Nn * Q), (1, Nn * Q), adjoint=adjoint)
        elif axis == 2:  # fibre (i, j): batch stride Q, element stride 1
            self.execute_strided(x, out, (Q, 1), (Q, 1), adjoint=adjoint)
        elif axis == 1:  # fibre (i, k): inner index k (stride 1), outer index i (stride Nn*Q), element stride Q
            self.execute_strided2(x, out, (1, Q, Nn * Q), (1, Q, Nn * Q), batch_inner=Q, adjoint=adjoint)
        else:
            raise ValueError("axis must be 0, 1 or 2")
        return out

    def table(self, which: int):
        sizes = {0: self.info["N"], 1: 2 * self.info["s"] * self.info["M"], 2: 2 * self.info["M"] ** 2,
                 3: self.info["n_c"] * self.info["M"] ** 2, 4: self.info["N"], 5: self.info["N"],
                 6: self.info["n_c"] * 484 // 2}
        with torch.cuda.device(self.device):
            # the table's own length when shorter (B(0): M^2; nodal P(0), P(1): 2 M^2)
            return B.lc_plan_table(self._handle, which, sizes[which], _stream_ptr(self.device))

    def autotune(self, x: torch.Tensor, out: torch.Tensor | None = None):
        """Pick the fastest chunk geometry on this input (see lc_plan_autotune)."""
        self._check_in(x)
        ib, ie = self._strides(x)
        if out is None:
            out = torch.empty_like(x)
        ob, oe = self._strides(out)
        with torch.cuda.device(self.device):
            return B.lc_plan_autotune(self._handle, x.data_ptr(), out.data_ptr(), ib, ie, ob, oe,
                                      _stream_ptr(self.device))

    def set_config(self, leaf_depth: int, chunk_depth: int):
        B.lc_plan_set_config(self._handle, leaf_depth, chunk_depth)

    def set_band(self, ctas: int = 0, after_leaf: bool = False):
        """Launch shape of the single-vector band (Step 6): CTAs (0 = one per group of
        strips) and whether it starts after the leaf restriction; results are unchanged."""
        B.lc_plan_set_band(self._handle, int(ctas), int(bool(after_leaf)))

    def set_split_schedule(self, persistent: bool = True):
        """Split tier: one persistent launch per execution (default) or one
        launch per level (results are bitwise the same)."""
        B.lc_plan_set_split_schedule(self._handle, int(bool(persistent)))

    def check(self):
        """Raise if a bounded device-side wait of an earlier execution ran out."""
        with torch.cuda.device(self.device):
            B.lc_plan_check(self._handle, _stream_ptr(self.device))

    def launches(self) -> int:
        return B.lc_plan_launches(self._handle)

    def close(self):
        if self._handle is not None:
            B.lc_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_PLAN_CACHE: dict = {}


def get_plan(n: int, direction: str, batch: int, dtype: str, device=None, **options) -> Plan:
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = (n, direction, batch, dtype, str(dev), tuple(sorted(options.items())))
    p = _PLAN_CACHE.get(key)
    if p is None:
        p = Plan(n, direction, batch, dtype, dev, **options)
        _PLAN_CACHE[key] = p
    return p


def leg2cheb(x: torch.Tensor, dtype: str | None = None, **options) -> torch.Tensor:
    """f_cheb = C^{-1} A f_leg along the last dimension of a 1-D or 2-D tensor."""
    dtype = dtype or ("f32" if x.dtype == torch.float32 else "f64")
    batch = 1 if x.dim() == 1 else x.shape[0]
    return get_plan(x.shape[-1], "l2c", batch, dtype, x.device, **options)(x)


def cheb2leg(x: torch.Tensor, dtype: str | None = None, **options) -> torch.Tensor:
    """f_leg = A^{-1} C f_cheb along the last dimension of a 1-D or 2-D tensor."""
    dtype = dtype or ("f32" if x.dtype == torch.float32 else "f64")
    batch = 1 if x.dim() == 1 else x.shape[0]
    return get_plan(x.shape[-1], "c2l", batch, dtype, x.device, **options)(x)


# -------------------------------------------------- leaf tile size autotuner
_TILE_CACHE: dict = {}


def autotune_tile(x: torch.Tensor, direction: str = "l2c", dtype: str = "f64_split", device=None, lengths=None,
                  n: int | None = None, batch: int = 1, candidates=(16, 20, 24, 28, 32), reps: int = 3,
                  **options):
    """Pick the leaf segment size s -- the tile every level inherits (level gamma
    works on blocks of h = s 2^(L-gamma-1) coefficients) -- for a plan shape by
    timing: one plan per candidate s (option fixed_s), `reps` executions on x
    each after a warm-up, the fastest kept.  Every s gives the same linear map;
    s changes the padding to N = s 2^(L+2), the number of levels and the block
    shapes.  Returns (plan, s, {s: ms per execution}).  The choice is cached
    per (lengths or (n, batch), direction, dtype) for later calls."""
    key = (tuple(int(v) for v in lengths) if lengths is not None else (int(n), int(batch)), direction, dtype)
    dev = torch.device(device) if device is not None else x.device
    if key in _TILE_CACHE:
        s = _TILE_CACHE[key][0]
        plan = Plan(n, direction, batch, dtype, dev, lengths=lengths, fixed_s=s, **options)
        return plan, s, dict(_TILE_CACHE[key][1])
    times = {}
    best = None
    for s in candidates:
        plan = Plan(n, direction, batch, dtype, dev, lengths=lengths, fixed_s=int(s), **options)
        out = torch.empty_like(x)
        plan(x, out=out)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan(x, out=out)
        e1.record()
        torch.cuda.synchronize(dev)
        times[int(s)] = e0.elapsed_time(e1) / reps
        if best is None or times[int(s)] < times[best[0]]:
            if best is not None:
                best[1].close()
            best = (int(s), plan)
        else:
            plan.close()
    _TILE_CACHE[key] = (best[0], dict(times))
    return best[1], best[0], times

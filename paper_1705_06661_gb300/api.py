"""Torch-facing API. PyTorch supplies device memory and streams only; every
step of the spin summation runs in the CUDA library behind the C-ABI.

Tensors use their own strides: dimension order is (spectators..., permuted...)
and any non-overlapping layout works. The fast layout is column-major with
the spectators fastest (``colmajor_empty``), i.e. A[a,b,c,i,j,k] stored with
a fastest, as in the paper's column-major convention (Sec. 3.1).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _binding as _b


def colmajor_empty(shape, dtype=torch.float64, device="cuda") -> torch.Tensor:
    """Dense column-major tensor (first index fastest) with logical shape `shape`."""
    shape = tuple(int(s) for s in shape)
    t = torch.empty(tuple(reversed(shape)), dtype=dtype, device=device)
    return t.permute(*reversed(range(len(shape))))


def colmajor_like(x: torch.Tensor) -> torch.Tensor:
    return colmajor_empty(x.shape, dtype=x.dtype, device=x.device)


def to_colmajor(x: torch.Tensor) -> torch.Tensor:
    y = colmajor_like(x)
    y.copy_(x)
    return y


def _coef_chain(coef, d: int) -> np.ndarray:
    c = np.asarray(coef.detach().cpu().numpy() if isinstance(coef, torch.Tensor) else coef, dtype=np.float64)
    if c.ndim == 1:
        c = c[None, :]
    if c.ndim != 2 or c.shape[1] != math.factorial(d):
        raise ValueError(f"coefficients must have shape [nfactors, {math.factorial(d)}]")
    return np.ascontiguousarray(c)


def _dims(x: torch.Tensor, d: int):
    """extents and element strides in ABI order (d spectators, d permuted);
    a tensor with only the d permuted dimensions gets spectator extents 1."""
    if x.dim() == 2 * d:
        return list(x.shape), list(x.stride())
    if x.dim() == d:
        return [1] * d + list(x.shape), [1] * d + list(x.stride())
    raise ValueError(f"expected a tensor with {d} or {2 * d} dimensions, got {x.dim()}")


def spinsum(A: torch.Tensor, coef, *, d: int | None = None, out: torch.Tensor | None = None,
            factorized: bool = False, adjoint: bool = False, strict: bool = False, tma: bool = False,
            alpha: float = 1.0, beta: float = 0.0, inplace: bool = False,
            stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """B = alpha * S(A) + beta * B (or A in place), S the spin summation of the
    coefficient chain `coef` ([nfactors, d!], lexicographic permutation order)."""
    if d is None:
        d = A.dim() // 2
    if d not in (2, 3, 4):
        raise ValueError("d must be 2, 3 or 4")
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if A.dtype == torch.float64:
        dtype = _b.SPINSUM_F64
    elif A.dtype == torch.float32:
        dtype = _b.SPINSUM_F32
    else:
        raise TypeError("A must be float64 or float32")
    c = _coef_chain(coef, d)
    if inplace:
        out = A
    elif out is None:
        out = colmajor_like(A) if beta == 0.0 else None
        if out is None:
            raise ValueError("beta != 0 needs an output tensor")
    if out.dtype != A.dtype or out.device != A.device or tuple(out.shape) != tuple(A.shape):
        raise ValueError("out must match A in dtype, device and shape")
    ext, lda = _dims(A, d)
    _, ldb = _dims(out, d)
    mode = (_b.SPINSUM_FACTORIZED if factorized else _b.SPINSUM_EXPANDED) | (_b.SPINSUM_ADJOINT if adjoint else 0) \
        | (_b.SPINSUM_STRICT if strict else 0) | (_b.SPINSUM_TMA if tma else 0)
    st = (stream or torch.cuda.current_stream(A.device)).cuda_stream
    fn = {2: _b.spinsum_2d, 3: _b.spinsum_3d, 4: _b.spinsum_4d}[d]
    with torch.cuda.device(A.device):
        fn(dtype, ext, A.data_ptr(), lda, out.data_ptr(), ldb, c, c.shape[0], mode, alpha, beta, int(inplace), st)
    return out


def contract(A: torch.Tensor, coef, W: torch.Tensor, *, d: int | None = None, out: torch.Tensor | None = None,
             factorized: bool = False, adjoint: bool = False, strict: bool = False,
             stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """C[s, y] = sum_t S(A)[s, t] * W[y, t] over the permuted group, with S(A)
    never stored (spinsum_contract); coef None contracts A itself. A: FP64,
    dense column-major (d spectators, d permuted indices). W: FP64, shape
    (Y, O**d), y fastest (a column-major copy is made otherwise). Returns C of
    shape (spectators..., Y), column-major (a new tensor unless `out` is one)."""
    if d is None:
        d = A.dim() // 2
    if A.dim() != 2 * d or A.dtype != torch.float64 or not A.is_cuda:
        raise ValueError("A must be a CUDA float64 tensor with 2d dimensions")
    ext, lda = _dims(A, d)
    dense = 1
    for k in range(2 * d):
        if ext[k] > 1 and lda[k] != dense:
            raise ValueError("A must be dense column-major")
        dense *= ext[k]
    T = int(np.prod(ext[d:]))
    if W.dim() != 2 or W.shape[1] != T or W.dtype != torch.float64 or W.device != A.device:
        raise ValueError(f"W must be a float64 tensor of shape (Y, {T}) on A's device")
    if W.stride(0) != 1 and W.shape[0] > 1:
        W = colmajor_empty(W.shape, device=A.device).copy_(W)
    Y = int(W.shape[0])
    ldw = int(W.stride(1)) if T > 1 else max(Y, 1)
    spec = tuple(A.shape[:d])
    S = int(np.prod(spec))
    if out is None:
        out = colmajor_empty(spec + (Y,), device=A.device)
    if tuple(out.shape) != spec + (Y,) or out.dtype != torch.float64:
        raise ValueError("out must have shape (spectators..., Y) and dtype float64")
    ldc = int(out.stride(-1)) if Y > 1 else max(S, 1)
    c = None if coef is None else _coef_chain(coef, d)
    mode = (_b.SPINSUM_FACTORIZED if factorized else _b.SPINSUM_EXPANDED) | (_b.SPINSUM_ADJOINT if adjoint else 0) \
        | (_b.SPINSUM_STRICT if strict else 0)
    st = (stream or torch.cuda.current_stream(A.device)).cuda_stream
    with torch.cuda.device(A.device):
        _b.spinsum_contract(d, ext, A.data_ptr(), c, 0 if c is None else c.shape[0], mode, W.data_ptr(), Y, ldw,
                            out.data_ptr(), ldc, st)
    return out


def spinsum_host(A: torch.Tensor, coef, *, out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                 d: int | None = None, factorized: bool = False, adjoint: bool = False, strict: bool = False,
                 alpha: float = 1.0, beta: float = 0.0, inplace: bool = False,
                 stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """The summation of a dense column-major CPU tensor (spinsum_3d_host /
    spinsum_4d_host). Pinned tensors are read and written by the kernel in
    place over the host link; pageable ones go through a three-stream
    copy-in / sum / copy-out pipeline in `workspace` (a CUDA byte tensor;
    default 3/8 of A's bytes, at least three slices). Asynchronous on `stream`:
    synchronize before reading `out`."""
    if d is None:
        d = A.dim() // 2
    if A.is_cuda:
        raise ValueError("A must be a CPU tensor")
    dtype = _b.SPINSUM_F64 if A.dtype == torch.float64 else _b.SPINSUM_F32
    c = _coef_chain(coef, d)
    if inplace:
        out = A
    elif out is None:
        out = colmajor_empty(A.shape, dtype=A.dtype, device="cpu")
    ext, lda = _dims(A, d)
    _, ldb = _dims(out, d)
    if workspace is None and A.is_pinned() and out.is_pinned():
        workspace = torch.empty(0, dtype=torch.uint8, device="cuda")   # zero-copy: no staging memory
    if workspace is None:
        slow = max(int(A.shape[d - 1]), 1)
        per = (A.numel() // slow) * A.element_size() * (2 if (beta != 0.0 and not inplace) else 1)
        nbytes = 3 * per * max(1, (slow + 7) // 8)
        workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    mode = (_b.SPINSUM_FACTORIZED if factorized else _b.SPINSUM_EXPANDED) | (_b.SPINSUM_ADJOINT if adjoint else 0) \
        | (_b.SPINSUM_STRICT if strict else 0)
    st = (stream or torch.cuda.current_stream(workspace.device)).cuda_stream
    fn = {2: _b.spinsum_2d_host, 3: _b.spinsum_3d_host, 4: _b.spinsum_4d_host}[d]
    with torch.cuda.device(workspace.device):
        fn(dtype, ext, A.data_ptr(), lda, out.data_ptr(), ldb, c, c.shape[0], mode, alpha, beta, int(inplace),
           workspace.data_ptr(), workspace.numel(), st)
    return out


def _dtype_code(x: torch.Tensor) -> int:
    if x.dtype == torch.float64:
        return _b.SPINSUM_F64
    if x.dtype == torch.float32:
        return _b.SPINSUM_F32
    raise ValueError("dtype must be float64 or float32")


def unpack(P: torch.Tensor, d: int, O: int, out: torch.Tensor | None = None,
           stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """Antisymmetric tensor B [spectators..., O, .., O] from its packed form P
    [spectators..., C(O, d)] (spinsum_unpack): B[s, t0 o tau] = sign(tau) P[s, r],
    r the colex rank of i_1 < .. < i_d; zero where an index repeats."""
    if not P.is_cuda:
        raise ValueError("P must be a CUDA tensor")
    nspec = P.dim() - 1
    if nspec != d:
        raise ValueError(f"P needs {d} spectator dimensions and the packed one")
    if P.shape[-1] != math.comb(O, d):
        raise ValueError(f"packed extent must be C({O}, {d}) = {math.comb(O, d)}")
    shape = tuple(P.shape[:d]) + (O,) * d
    if out is None:
        out = colmajor_empty(shape, dtype=P.dtype, device=P.device)
    st = (stream or torch.cuda.current_stream(P.device)).cuda_stream
    _b.spinsum_unpack(d, _dtype_code(P), list(shape), P.data_ptr(), list(P.stride()), out.data_ptr(),
                      list(out.stride()), st)
    return out


def pack(B: torch.Tensor, d: int, out: torch.Tensor | None = None,
         stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """Packed form P [spectators..., C(O, d)] of an antisymmetric tensor B
    [spectators..., O, .., O] (spinsum_pack): P[s, r] = B[s, i_1 < .. < i_d]."""
    if not B.is_cuda:
        raise ValueError("B must be a CUDA tensor")
    if B.dim() != 2 * d:
        raise ValueError(f"B needs {2 * d} dimensions")
    O = int(B.shape[d])
    if out is None:
        out = colmajor_empty(tuple(B.shape[:d]) + (math.comb(O, d),), dtype=B.dtype, device=B.device)
    st = (stream or torch.cuda.current_stream(B.device)).cuda_stream
    _b.spinsum_pack(d, _dtype_code(B), list(B.shape), B.data_ptr(), list(B.stride()), out.data_ptr(),
                    list(out.stride()), st)
    return out


class SpinSumFunction(torch.autograd.Function):
    """Differentiable spin summation. The operator is linear, so the gradient
    of B = alpha S(A) is alpha S^T(gB), S^T = sum a_sigma pi_{sigma^-1} for one
    factor and F_k^T ... F_1^T for a chain; the backward pass is the same orbit
    kernel with SPINSUM_ADJOINT."""

    @staticmethod
    def forward(ctx, A, coef, d, factorized, alpha):
        ctx.coef, ctx.d, ctx.factorized, ctx.alpha = coef, d, factorized, alpha
        return spinsum(A, coef, d=d, factorized=factorized, alpha=alpha)

    @staticmethod
    def backward(ctx, gB):
        gA = spinsum(gB, ctx.coef, d=ctx.d, factorized=ctx.factorized, adjoint=True, alpha=ctx.alpha)
        return gA, None, None, None, None


def spinsum_autograd(A: torch.Tensor, coef, *, d: int | None = None, factorized: bool = False,
                     alpha: float = 1.0) -> torch.Tensor:
    d = d if d is not None else A.dim() // 2
    return SpinSumFunction.apply(A, _coef_chain(coef, d), d, factorized, float(alpha))


class Plan:
    """Batched spin summations run by one persistent kernel launch per
    (d, arithmetic) class (spinsum_plan_create / _execute / _destroy).

    problems: list of dicts with keys A, coef and optionally B (output; None
    means in place), d, factorized, adjoint, strict, alpha, beta. All tensors
    share one dtype. tune=True lets the autotuner time candidate tilings
    (which runs the problems); tune=False uses the heuristic."""

    def __init__(self, problems, tune: bool = True, stream: torch.cuda.Stream | None = None):
        self._keep = []
        structs = []
        dtypes = set()
        for p in problems:
            A = p["A"]
            d = p.get("d", A.dim() // 2)
            B = p.get("B")
            inplace = B is None
            out = A if inplace else B
            c = _coef_chain(p["coef"], d)
            ext, lda = _dims(A, d)
            _, ldb = _dims(out, d)
            mode = (_b.SPINSUM_FACTORIZED if p.get("factorized") else 0) | (
                _b.SPINSUM_ADJOINT if p.get("adjoint") else 0) | (_b.SPINSUM_STRICT if p.get("strict") else 0)
            s = _b.spinsum_problem()
            s.d = d
            for k in range(2 * d):
                s.ext[k], s.lda[k], s.ldb[k] = int(ext[k]), int(lda[k]), int(ldb[k])
            s.A, s.B = A.data_ptr(), out.data_ptr()
            s.coef = c.ctypes.data
            s.nfactors = c.shape[0]
            s.mode = mode
            s.alpha, s.beta = float(p.get("alpha", 1.0)), float(p.get("beta", 0.0))
            s.inplace = int(inplace)
            structs.append(s)
            self._keep += [A, out, c]
            dtypes.add(A.dtype)
        if len(dtypes) > 1:
            raise ValueError("all problems of a plan share one dtype")
        dt = dtypes.pop() if dtypes else torch.float64
        self.dtype = _b.SPINSUM_F64 if dt == torch.float64 else _b.SPINSUM_F32
        dev = problems[0]["A"].device if problems else torch.device("cuda")
        st = (stream or torch.cuda.current_stream(dev)).cuda_stream
        with torch.cuda.device(dev):
            self._h = _b.spinsum_plan_create(structs, self.dtype, int(tune), st)
        self.device = dev

    def execute(self, stream: torch.cuda.Stream | None = None) -> None:
        st = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        _b.spinsum_plan_execute(self._h, st)

    def describe(self) -> str:
        return _b.spinsum_plan_describe(self._h)

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _b.spinsum_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

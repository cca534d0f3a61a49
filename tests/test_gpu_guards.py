"""No kernel writes outside its output: every tensor lives inside a larger
buffer whose other elements (guard zones before and after, and the gaps of
strided layouts) hold a sentinel bit pattern, which must survive the call
bit for bit; an out-of-place call must leave A's whole buffer unchanged; and
the result must match the oracle. One case per kernel path and edge: the
orbit-stream kernel with 16-byte and with misaligned (scalar) runs, odd
spectator blocks, 4D, FP32, in place and with beta; the tiled kernel on
ragged N^3 / N^4 tensors with paired and with scalar copies; the general-
stride kernel; and a batched plan."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_within, fp32_tol, fp64_tol

pytestmark = pytest.mark.gpu

SENT64 = 0x7FF8DEADBEEF0123
SENT32 = 0x7FC0BEEF


def _guarded(A_np, tdt, guard, strides=None):
    """A buffer with `guard` sentinel elements on each side of the tensor, the
    tensor stored with the given element strides (column-major dense by
    default); returns (buffer, tensor view, mask of the tensor's elements)."""
    import torch
    shape = A_np.shape
    if strides is None:
        strides, s = [], 1
        for e in shape:
            strides.append(s)
            s *= e
    span = 1 + sum((e - 1) * st for e, st in zip(shape, strides)) if A_np.size else 0
    n = span + 2 * guard
    buf = torch.empty(n, dtype=tdt, device="cuda")
    ibuf = buf.view(torch.int64 if tdt == torch.float64 else torch.int32)
    ibuf.fill_(SENT64 if tdt == torch.float64 else SENT32)
    t = buf.as_strided(shape, strides, guard)
    t.copy_(torch.from_numpy(A_np).to(tdt).cuda())
    idx = torch.arange(n).as_strided(shape, strides, guard)
    mask = np.zeros(n, dtype=bool)
    mask[idx.reshape(-1).numpy()] = True
    return buf, t, mask


def _check_guards(buf, mask, msg):
    import torch
    ib = buf.view(torch.int64 if buf.dtype == torch.float64 else torch.int32).cpu().numpy()
    sent = SENT64 if buf.dtype == torch.float64 else SENT32
    outside = ib[~mask]
    bad = np.nonzero(outside != np.array(sent, dtype=ib.dtype))[0]
    assert bad.size == 0, f"{msg}: {bad.size} elements outside the tensor were written"


CASES = [
    # name, d, shape, coef row (0: random set, -1: the d = 2 set 2, -1), factorized, dtype, guard, strides-kind
    ("k1 3d 16-byte runs", 3, (6, 6, 6, 8, 8, 8), 1, True, "f64", 4096, None),
    ("k1 3d misaligned runs", 3, (6, 6, 6, 8, 8, 8), 1, True, "f64", 4097, None),
    ("k1 3d odd spectator block", 3, (5, 5, 5, 7, 7, 7), 2, False, "f64", 4096, None),
    ("k1 4d", 4, (4, 4, 4, 4, 6, 6, 6, 6), 5, True, "f64", 4096, None),
    ("k1 4d random set", 4, (3, 3, 3, 3, 7, 7, 7, 7), 0, False, "f64", 4097, None),
    ("k1 3d fp32", 3, (6, 6, 6, 8, 8, 8), 1, True, "f32", 4096, None),
    ("k1 3d fp32 misaligned", 3, (6, 6, 6, 8, 8, 8), 1, True, "f32", 4099, None),
    ("k2 3d ragged", 3, (21, 21, 21), 1, True, "f64", 4096, None),
    ("k2 3d ragged scalar copies", 3, (19, 19, 19), 1, True, "f64", 4097, None),
    ("k2 4d ragged", 4, (9, 9, 9, 9), 6, True, "f64", 4096, None),
    ("k2 4d fp32", 4, (10, 10, 10, 10), 5, True, "f32", 4096, None),
    ("kg sliced spectators", 3, (4, 4, 4, 6, 6, 6), 1, True, "f64", 4096, "gaps"),
    ("k1 2d", 2, (24, 24, 20, 20), -1, False, "f64", 4096, None),
    ("k1 2d misaligned", 2, (24, 24, 20, 20), -1, False, "f64", 4097, None),
    ("k2 2d ragged", 2, (70, 70), -1, False, "f64", 4096, None),
    ("k2 2d ragged scalar copies", 2, (45, 45), -1, False, "f32", 4097, None),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode", ["out", "inplace", "beta"])
def test_writes_stay_inside(case, mode):
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    name, d, shape, row, fac, dt, guard, sk = case
    tdt = torch.float64 if dt == "f64" else torch.float32
    coef = np.array([[2.0, -1.0]]) if row < 0 else (wl.table2(row) if row else wl.random_coef(d, 77))
    A_np = wl.uniform(31, shape)
    if dt == "f32":
        A_np = A_np.astype(np.float32).astype(np.float64)
    strides = None
    if sk == "gaps":                     # every index at twice its dense stride, then + 1 on the first
        strides, s = [], 1
        for e in shape:
            strides.append(2 * s)
            s *= e
        strides[0] = 2
    abuf, A, amask = _guarded(A_np, tdt, guard, strides)
    alpha, beta = (0.5, -1.25) if mode == "beta" else (1.0, 0.0)
    B0_np = wl.uniform(32, shape)
    if dt == "f32":
        B0_np = B0_np.astype(np.float32).astype(np.float64)
    if mode == "inplace":
        ss.spinsum(A, coef, d=d, inplace=True, factorized=fac, alpha=alpha, beta=beta)
        got, buf, mask = A, abuf, amask
        bold = A_np
    else:
        bbuf, B, bmask = _guarded(B0_np, tdt, guard + 2, strides)
        a_before = abuf.clone()
        ss.spinsum(A, coef, d=d, out=B, factorized=fac, alpha=alpha, beta=beta)
        torch.cuda.synchronize()
        assert torch.equal(abuf.view(torch.int64 if tdt == torch.float64 else torch.int32),
                           a_before.view(torch.int64 if tdt == torch.float64 else torch.int32)), f"{name}: A written"
        got, buf, mask = B, bbuf, bmask
        bold = B0_np
    torch.cuda.synchronize()
    ss.spinsum_check_status(torch.cuda.current_stream().cuda_stream)
    _check_guards(buf, mask, name)
    want = alpha * oracle.spinsum(A_np, d, coef, factorized=fac) + (beta * bold if beta else 0.0)
    res = got.double().cpu().numpy()
    tol = fp64_tol(d, coef, fac, A_np, alpha) if dt == "f64" else fp32_tol(d, coef, fac, A_np) * 2
    tol += (abs(beta) * np.abs(bold).max() * 2.0 ** (-52 if dt == "f64" else -23)) if beta else 0.0
    assert_within(res, want, tol, name)


def test_batched_plan_writes_stay_inside():
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    shapes = [(7, 7, 7, 6, 6, 6), (8, 8, 8, 9, 9, 9), (5, 5, 5, 11, 11, 11)]
    specs, keep = [], []
    for i, shp in enumerate(shapes):
        A_np = wl.uniform(40 + i, shp)
        abuf, A, amask = _guarded(A_np, torch.float64, 4096 + i)
        bbuf, B, bmask = _guarded(np.zeros(shp), torch.float64, 4099 + i)
        coef = wl.table2(1 + i)
        specs.append({"A": A, "B": B, "coef": coef, "d": 3, "factorized": True})
        keep.append((A_np, coef, bbuf, bmask, B))
    plan = ss.Plan(specs, tune=False)
    plan.execute()
    torch.cuda.synchronize()
    for A_np, coef, bbuf, bmask, B in keep:
        _check_guards(bbuf, bmask, "batched")
        want = oracle.spinsum(A_np, 3, coef, factorized=True)
        assert_within(B.cpu().numpy(), want, fp64_tol(3, coef, True, A_np), "batched")
    plan.close()

"""spinsum_batch_static: the batched summation for callers that cannot
allocate device memory (codes that reserve HBM up front and hand it out only
from their own pool, or services that may not call cudaMalloc on a request
path). It keeps its parameters in a fixed device array of the library.

Checked here through the C-ABI against the existing batched entry point
(a plan), on two calls in a row with different problem sets, so that a
stale array from the first call would show up in the second. This file sorts
last so that a stopping test run has already run every other test."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_within, fp64_tol

pytestmark = pytest.mark.gpu


def _make(seed, shapes):
    import torch
    import paper_1705_06661_gb300 as ss
    probs = []
    for k, (d, shape, coef, fac) in enumerate(shapes):
        A_np = wl.uniform(seed + k, shape)
        A = ss.to_colmajor(torch.from_numpy(A_np).cuda())
        probs.append({"A": A, "A_np": A_np, "d": d, "coef": coef, "factorized": fac,
                      "B_plan": ss.colmajor_like(A), "B_static": ss.colmajor_like(A)})
    return probs


def _struct(p, out):
    import paper_1705_06661_gb300 as ss
    from paper_1705_06661_gb300 import api
    d = p["d"]
    c = api._coef_chain(p["coef"], d)
    ext, lda = api._dims(p["A"], d)
    _, ldb = api._dims(out, d)
    s = ss.spinsum_problem()
    s.d = d
    for k in range(2 * d):
        s.ext[k], s.lda[k], s.ldb[k] = int(ext[k]), int(lda[k]), int(ldb[k])
    s.A, s.B = p["A"].data_ptr(), out.data_ptr()
    s.coef = c.ctypes.data
    s.nfactors = c.shape[0]
    s.mode = ss.SPINSUM_FACTORIZED if p["factorized"] else 0
    s.alpha, s.beta, s.inplace = 1.0, 0.0, 0
    return s, c


def _run_both(probs):
    import torch
    import paper_1705_06661_gb300 as ss
    st = torch.cuda.current_stream().cuda_stream
    keep = []
    plan_structs, static_structs = [], []
    for p in probs:
        s1, c1 = _struct(p, p["B_plan"])
        s2, c2 = _struct(p, p["B_static"])
        keep += [c1, c2]
        plan_structs.append(s1)
        static_structs.append(s2)
    h = ss.spinsum_plan_create(plan_structs, ss.SPINSUM_F64, 0, st)
    ss.spinsum_plan_execute(h, st)
    ss.spinsum_batch_static(static_structs, ss.SPINSUM_F64, st)
    torch.cuda.synchronize()
    ss.spinsum_check_status(st)
    ss.spinsum_plan_destroy(h)
    for p in probs:
        got = p["B_static"].cpu().numpy()
        want = p["B_plan"].cpu().numpy()
        assert_within(got, want, fp64_tol(p["d"], p["coef"], p["factorized"], p["A_np"]), "static vs plan")


def test_static_batch_matches_plan_on_two_calls():
    first = _make(700, [
        (3, (6, 5, 7, 5, 5, 5), wl.table2(1), True),      # odd spectator block: scalar path
        (3, (8, 8, 8, 6, 6, 6), wl.random_coef(3, 701), False),
        (4, (3, 3, 3, 3, 5, 5, 5, 5), wl.table2(5), True),
        (3, (4, 4, 4, 3, 3, 3), wl.table2(2), False),
    ])
    _run_both(first)
    # a second call with other problems: nothing of the first may leak into it
    second = _make(800, [
        (4, (2, 2, 2, 2, 6, 6, 6, 6), wl.random_coef(4, 801), False),
        (3, (10, 10, 10, 4, 4, 4), wl.table2(3), False),
    ])
    _run_both(second)


def test_static_batch_rejects_too_many_problems():
    import torch
    import paper_1705_06661_gb300 as ss
    p = _make(900, [(3, (4, 4, 4, 3, 3, 3), wl.table2(1), False)])[0]
    s, c = _struct(p, p["B_static"])
    with pytest.raises(ss.SpinsumError, match="at most 64"):
        ss.spinsum_batch_static([s] * (ss.SPINSUM_STATIC_MAX_PROBLEMS + 1), ss.SPINSUM_F64,
                                torch.cuda.current_stream().cuda_stream)

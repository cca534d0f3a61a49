"""spinsum_batch_static: the batched summation for callers that cannot
allocate device memory (codes that reserve HBM up front and hand it out only
from their own pool, or services that may not call cudaMalloc on a request
path). It keeps its parameters in a fixed device array of the library.

Checked here through the C-ABI, on two calls in a row with different problem
sets (so that a stale array from the first call would show up in the second):
against the oracle directly, and against the existing batched entry point (a
plan). Also checked: device free memory does not move across repeated calls,
more than 64 problems are refused, and a stream that is being captured is
refused (the parameter upload reads a host buffer that lives only for the
call). This file sorts last so that a stopping test run has already run every
other test."""
import numpy as np
import pytest

import oracle
import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, fp64_tol

pytestmark = pytest.mark.gpu


def _make(seed, shapes, integer=False):
    import torch
    import paper_1705_06661_gb300 as ss
    probs = []
    for k, (d, shape, coef, fac) in enumerate(shapes):
        A_np = wl.integers(seed + k, shape) if integer else wl.uniform(seed + k, shape)
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


def _run_both(probs, integer=False):
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
        want = oracle.spinsum(p["A_np"], p["d"], p["coef"], factorized=p["factorized"])
        if integer:
            assert_bitexact(got, want, "static vs oracle")
        else:
            assert_within(got, want, fp64_tol(p["d"], p["coef"], p["factorized"], p["A_np"]), "static vs oracle")
        assert_within(got, p["B_plan"].cpu().numpy(),
                      fp64_tol(p["d"], p["coef"], p["factorized"], p["A_np"]), "static vs plan")


FIRST = [
    (3, (6, 5, 7, 5, 5, 5), wl.table2(1), True),      # odd spectator block: scalar path
    (3, (8, 8, 8, 6, 6, 6), wl.random_coef(3, 701), False),
    (4, (3, 3, 3, 3, 5, 5, 5, 5), wl.table2(5), True),
    (3, (4, 4, 4, 3, 3, 3), wl.table2(2), False),
]
SECOND = [
    (4, (2, 2, 2, 2, 6, 6, 6, 6), wl.random_coef(4, 801), False),
    (3, (10, 10, 10, 4, 4, 4), wl.table2(3), False),
]


def test_static_batch_matches_oracle_and_plan_on_two_calls():
    _run_both(_make(700, FIRST))
    # a second call with other problems: nothing of the first may leak into it
    _run_both(_make(800, SECOND))


def test_static_batch_integer_inputs_bit_exact():
    _run_both(_make(710, FIRST, integer=True), integer=True)
    _run_both(_make(810, SECOND, integer=True), integer=True)


def test_static_batch_allocates_no_device_memory():
    import torch
    import paper_1705_06661_gb300 as ss
    probs = _make(720, FIRST)
    structs, keep = [], []
    for p in probs:
        s, c = _struct(p, p["B_static"])
        structs.append(s)
        keep.append(c)
    st = torch.cuda.current_stream().cuda_stream
    ss.spinsum_batch_static(structs, ss.SPINSUM_F64, st)   # warm-up: loads the kernels
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        ss.spinsum_batch_static(structs, ss.SPINSUM_F64, st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory moved by {free0 - free1} bytes across calls"
    ss.spinsum_check_status(st)


def test_static_batch_rejects_too_many_problems():
    import torch
    import paper_1705_06661_gb300 as ss
    p = _make(900, [(3, (4, 4, 4, 3, 3, 3), wl.table2(1), False)])[0]
    s, c = _struct(p, p["B_static"])
    with pytest.raises(ss.SpinsumError, match="at most 64"):
        ss.spinsum_batch_static([s] * (ss.SPINSUM_STATIC_MAX_PROBLEMS + 1), ss.SPINSUM_F64,
                                torch.cuda.current_stream().cuda_stream)


def test_static_batch_refuses_a_capturing_stream():
    import torch
    import paper_1705_06661_gb300 as ss
    p = _make(910, [(3, (4, 4, 4, 3, 3, 3), wl.table2(1), False)])[0]
    s, c = _struct(p, p["B_static"])
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    raised = None
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        g.capture_begin()
        try:
            ss.spinsum_batch_static([s], ss.SPINSUM_F64, side.cuda_stream)
        except ss.SpinsumError as e:
            raised = e
        finally:
            g.capture_end()
    from paper_1705_06661_gb300 import _binding
    assert raised is not None and raised.status == _binding.SPINSUM_ERR_ARG and "captured" in str(raised)
    # the same call outside capture still runs
    ss.spinsum_batch_static([s], ss.SPINSUM_F64, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert_within(p["B_static"].cpu().numpy(), oracle.spinsum(p["A_np"], 3, p["coef"]),
                  fp64_tol(3, p["coef"], False, p["A_np"]), "after refusal")

"""The allocation-free entry point (mr_run_static) against the context path.

mr_run_static is for callers that cannot allocate device memory when they run
a problem; it works inside a scratch area built into the library.  This file
is collected last so that a failure here stops a -x run only after every other
test has run; it passes alone in a fresh process as well as after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64, capi, workloads as W
from paper_2102_12163_gb300 import _desc as desc_of

pytestmark = pytest.mark.gpu

CASES = [
    ("burgers-copy-J11", lambda: W.random_smooth(11, W.EQ_BURGERS, seed=71, eps=1e-4, bc=W.BC_COPY), MR_FP64),
    ("euler-periodic-J12", lambda: W.random_smooth(12, W.EQ_EULER, seed=72, eps=1e-4), MR_FP64),
    ("sw-copy-J10-fp32", lambda: W.random_smooth(10, W.EQ_SW, seed=73, eps=1e-4, bc=W.BC_COPY), MR_FP32_MIXED),
]


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("name,make,precision", CASES, ids=[c[0] for c in CASES])
def test_static_scratch_matches_the_context_path(torch_cuda, name, make, precision):
    torch = torch_cuda
    from paper_2102_12163_gb300 import MRLBM

    L = capi.load()
    inst = make()
    steps = 25
    # existing entry points: context with a caller-allocated workspace
    s = MRLBM(inst, precision=precision)
    s.set_initial()
    s.advance(steps)
    ref = s.finest()
    ref_updates = s.stats()[0]
    # allocation-free entry point, twice in a row on the same inputs
    d = desc_of(inst)
    m = torch.as_tensor(np.ascontiguousarray(inst.m0, dtype=np.float64)).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((inst.nf, 1 << inst.Jmax), float("nan"), dtype=torch.float64, device="cuda")
        upd = ctypes.c_ulonglong()
        rc = L.mr_run_static(ctypes.byref(d), precision, ctypes.c_void_p(m.data_ptr()), steps,
                             ctypes.c_void_p(out.data_ptr()), ctypes.byref(upd), ctypes.c_void_p(stream.cuda_stream))
        capi.check(None, rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12, (call, float(np.max(np.abs(got - ref))))
        assert upd.value == ref_updates


def test_static_scratch_rejects_instances_beyond_its_size(torch_cuda):
    L = capi.load()
    inst = W.random_smooth(8, W.EQ_EULER, seed=74)
    d = desc_of(inst)
    d.Jmax = 20  # layout far beyond MR_STATIC_SCRATCH_BYTES
    rc = L.mr_run_static(ctypes.byref(d), MR_FP64, ctypes.c_void_p(1), 1, ctypes.c_void_p(1), None, None)
    assert rc == capi.MR_ERR_CAPACITY
    buf = ctypes.create_string_buffer(256)
    L.mr_last_error(None, buf, 256)
    assert b"static area" in buf.value

"""wproj_phi_noalloc, the forward operator for callers that cannot allocate
device memory (their memory belongs to another runtime's pool, or their loop
cannot take cudaMalloc's device-wide synchronisation).  Called through the
C-ABI, it must give the same visibilities as wproj_phi on consecutive calls,
and refuse a plan whose scratch would not fit its fixed array.

This file is named to be collected last, so that a run stopping at the first
failure has run every other test before it."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


# index formats (their partial-sum counts, and so the scratch layout, differ),
# 16-bit values with row scales, and the paper's operator, whose upsampling
# step uses the FFT slot of the scratch as 2 N^2 work
CASES = [
    dict(id="auto-f32", N=64, M=1229, kw={}),
    dict(id="columns-f32", N=64, M=1229, kw=dict(index_format="columns")),
    dict(id="mask-f32", N=64, M=600, kw=dict(index_format="mask")),
    dict(id="columns-bf16", N=64, M=1229, kw=dict(index_format="columns", value_dtype="bf16")),
    dict(id="mask-bf16", N=32, M=400, kw=dict(index_format="mask", value_dtype="bf16")),
    dict(id="paper-mode", N=32, M=None, kw=dict(kb_support=1, chirp="linear", upsampling=True)),
    dict(id="runs-f32", N=32, M=500, wd=0.2, kw=dict(index_format="runs")),
    dict(id="runs-bf16", N=64, M=800, wd=0.05, kw=dict(index_format="runs", value_dtype="bf16", box=32)),
]


@pytest.mark.parametrize("case", CASES, ids=[c["id"] for c in CASES])
def test_phi_noalloc_matches_phi_on_consecutive_calls(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_3424_gb300 import synth, wproj
    dev = torch.device("cuda", torch.cuda.current_device())
    L = synth.fov_L()
    N = case["N"]
    rng = np.random.default_rng(11)
    if case["M"] is None:
        uvw = synth.paper_problem(N, 0.2, seed=2).uvw
    else:
        # run lengths need kernels that fit their box: small w for those cases
        uvw = synth.random_uvw(rng, case["M"], N, L, case.get("wd", 1.0))
    M = uvw.shape[0]
    plan = wproj.Plan(N, L, **case["kw"])
    plan.build_kernels(torch.from_numpy(uvw).to(dev), 0.99)
    lib = wproj.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        x = torch.from_numpy(rng.standard_normal((N, N)).astype(np.float32)).to(dev)
        y_ref = torch.empty(M, dtype=torch.complex64, device=dev)
        y_new = torch.full((M,), float("nan"), dtype=torch.complex64, device=dev)
        assert lib.wproj_phi(plan.handle, _vp(x), _vp(y_ref), stream) == wproj.OK
        assert lib.wproj_phi_noalloc(plan.handle, _vp(x), _vp(y_new), stream) == wproj.OK, \
            lib.wproj_last_error().decode()
        torch.cuda.synchronize()
        rel = (torch.linalg.vector_norm(y_new - y_ref) / torch.linalg.vector_norm(y_ref)).item()
        assert rel <= 1e-5, (call, rel)
    plan.close()


def test_phi_noalloc_rejects_a_plan_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_3424_gb300 import synth, wproj
    dev = torch.device("cuda", torch.cuda.current_device())
    L = synth.fov_L()
    N = 1024                        # the padded spectrum alone is 32 MiB
    plan = wproj.Plan(N, L, box=16)
    plan.build_kernels(torch.zeros((1, 3), dtype=torch.float64, device=dev), 0.99)
    x = torch.zeros((N, N), dtype=torch.float32, device=dev)
    y = torch.empty(1, dtype=torch.complex64, device=dev)
    lib = wproj.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.wproj_phi_noalloc(plan.handle, _vp(x), _vp(y), stream) == wproj.ERR_INVALID_ARG
    assert b"limit" in lib.wproj_last_error()
    plan.close()

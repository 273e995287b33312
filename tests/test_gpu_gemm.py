"""The tcgen05 BF16 GEMM (C = A B^T + bias, FP32 accumulation) against a plain
FP64 CPU product of the same BF16 inputs."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1307_3424_gb300 import wproj
    return wproj


@pytest.mark.parametrize("m,n,k,bias,out_bf16", [(128, 128, 64, False, False), (256, 384, 128, True, False),
                                                 (512, 256, 256, True, False), (128, 3072, 256, True, True),
                                                 (1024, 256, 1024, False, False)])
def test_gemm_matches_cpu(wp, m, n, k, bias, out_bf16):
    g = torch.Generator().manual_seed(m + n + k)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    bs = torch.randn(n, generator=g) if bias else None
    ref = a.double() @ b.double().T
    if bias:
        ref = ref + bs.double()
    c = wp.gemm_bf16(a.cuda(), b.cuda(), bs.cuda() if bias else None, out_bf16=out_bf16).cpu().double()
    err = float((c - ref).norm() / ref.norm())
    assert err <= (4e-3 if out_bf16 else 1e-5), err


def test_gemm_structure(wp):
    # unit vectors locate every (row, column) of the tile: C = A B^T picks entries
    m, n, k = 256, 128, 128
    a = torch.zeros(m, k)
    b = torch.zeros(n, k)
    for i in range(m):
        a[i, i % k] = 1.0 + (i // k)
    for j in range(n):
        b[j, (3 * j) % k] = 1.0
    ref = a @ b.T
    c = wp.gemm_bf16(a.to(torch.bfloat16).cuda(), b.to(torch.bfloat16).cuda()).cpu()
    assert torch.equal(c, ref)


def test_gemm_rejects_bad_shapes(wp):
    a = torch.zeros(100, 64, dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(wp.WprojError):
        wp.gemm_bf16(a, b)


def test_gemm_wait_timeout_is_reported_and_the_context_recovers(wp):
    # the test hook makes every CTA wait on an mbarrier nothing arrives on, for
    # 1 ms: the call must report the timeout (no fault, no hang), and the next
    # call, with the hook off, must give the right product
    g = torch.Generator().manual_seed(3)
    a = torch.randn(256, 256, generator=g).to(torch.bfloat16)
    b = torch.randn(128, 256, generator=g).to(torch.bfloat16)
    lib = wp.lib()
    assert lib.wproj_gemm_test_hook(1, 1_000_000) == wp.OK
    try:
        with pytest.raises(wp.WprojError) as ei:
            wp.gemm_bf16(a.cuda(), b.cuda())
        assert ei.value.status == wp.ERR_TIMEOUT
        assert b"wait ran out" in lib.wproj_last_error()
    finally:
        assert lib.wproj_gemm_test_hook(0, 0) == wp.OK
    c = wp.gemm_bf16(a.cuda(), b.cuda()).cpu().double()
    ref = a.double() @ b.double().T
    assert float((c - ref).norm() / ref.norm()) <= 1e-5

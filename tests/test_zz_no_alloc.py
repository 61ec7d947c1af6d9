"""The non-allocating fgemm entry point (fgemm_modp_noalloc).

fgemm_modp_noalloc is for callers that may not allocate device memory: a
component that runs inside another one's memory pool, or a latency-critical
path that must not meet the device synchronisation an allocation can bring.
It keeps its digit planes in a fixed device array inside the library instead
of context workspace.  Two calls in a row (the second reusing the array as the
first left it) must each give exactly C - A B mod p, checked against an exact
host product and against the allocating entry point, for every digit count
(L = 1..4: p = 251, 65521 / 131071, 1048573, 2^31 - 1), for p = 2 and for
strided views.  This file is collected last so that a failure here does not
hide the other tests; it also passes alone in a fresh process, where its first
call performs the per-device set-up.
"""
import numpy as np
import pytest

from pluq_checks import matmul_mod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1402_3501_gb300 as pq  # noqa: E402
from paper_1402_3501_gb300 import binding  # noqa: E402


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(X).astype(np.int64).astype(np.int32)).cuda()


def _exact(C, A, B, p):
    return (C.astype(np.int64) - matmul_mod(A, B, p)) % p


@pytest.mark.parametrize("p", [2, 251, 65521, 131071, 1048573, 2147483647])
def test_noalloc_exact_twice(p):
    rng = np.random.default_rng(p % 1000 + 7)
    ctx = pq.Context(0)
    try:
        for (M, N, K) in [(300, 200, 700), (129, 257, 1030)]:
            A = rng.integers(0, p, (M, K), dtype=np.int64)
            B = rng.integers(0, p, (K, N), dtype=np.int64)
            C = rng.integers(0, p, (M, N), dtype=np.int64)
            A[0, :] = p - 1  # the largest digit products the exact blocks absorb
            B[:, 0] = p - 1
            expect = _exact(C, A, B, p)
            got = pq.fgemm_modp_noalloc(_dev(C), _dev(A), _dev(B), p)
            want = pq.fgemm_modp(_dev(C), _dev(A), _dev(B), p, form="limb", ctx=ctx)
            torch.cuda.synchronize()
            assert np.array_equal(got.cpu().numpy().astype(np.int64) % (1 << 32), expect)
            assert torch.equal(got, want)
    finally:
        ctx.close()


@pytest.mark.parametrize("p", [131071, 2147483647])
def test_noalloc_strided_views(p):
    rng = np.random.default_rng(5)
    big = _dev(rng.integers(0, p, (300, 400), dtype=np.int64))
    A = big[10:110, 5:77]
    B = big[120:192, 200:333]
    for _ in range(2):
        C = big[200:300, 0:133].clone()
        expect = _exact(C.cpu().numpy().astype(np.int64) % (1 << 32),
                        A.cpu().numpy().astype(np.int64) % (1 << 32),
                        B.cpu().numpy().astype(np.int64) % (1 << 32), p)
        pq.fgemm_modp_noalloc(C, A, B, p)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy().astype(np.int64) % (1 << 32), expect)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    p = 131071
    A = torch.zeros((4096, 4096), dtype=torch.int32, device="cuda")
    with pytest.raises(pq.PluqError) as e:
        pq.fgemm_modp_noalloc(A.clone(), A, A, p)
    assert e.value.status == -9
    # one huge inner dimension is refused before any byte count is formed
    a = torch.zeros((1, 1), dtype=torch.int32, device="cuda")
    st = pq.load().fgemm_modp_noalloc(p, 1, 1, 1 << 40, binding._dev_ptr(a), 1 << 40,
                                      binding._dev_ptr(a), 1, binding._dev_ptr(a), 1, None)
    assert st == -9

"""The non-allocating fgemm entry point (fgemm_modp_noalloc) against fgemm_modp.

fgemm_modp_noalloc serves callers that cannot allocate device memory; it
keeps its digit planes in a fixed device array inside the library.  Two calls
in a row (the second reusing the array left by the first) must give exactly
the results of the allocating entry point.  This file is collected last so
that a failure here does not hide the other tests; it passes alone in a
fresh process too (the first call then performs the per-device set-up).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1402_3501_gb300 as pq  # noqa: E402


def _rand(rng, shape, p):
    return torch.from_numpy(rng.integers(0, p, shape, dtype=np.int64).astype(np.int32)).cuda()


@pytest.mark.parametrize("p", [131071, 65521, 251])
def test_noalloc_matches_fgemm_modp_twice(p):
    rng = np.random.default_rng(p)
    ctx = pq.Context(0)
    for (M, N, K) in [(300, 200, 700), (129, 257, 1030)]:
        A, B, C = _rand(rng, (M, K), p), _rand(rng, (K, N), p), _rand(rng, (M, N), p)
        want = pq.fgemm_modp(C.clone(), A, B, p, form="limb", ctx=ctx)
        got = pq.fgemm_modp_noalloc(C.clone(), A, B, p)
        torch.cuda.synchronize()
        assert torch.equal(got, want)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    p = 131071
    A = torch.zeros((4096, 4096), dtype=torch.int32, device="cuda")
    with pytest.raises(pq.PluqError) as e:
        pq.fgemm_modp_noalloc(A.clone(), A, A, p)
    assert e.value.status == -9

"""Failure detection without a GPU fault: a specialised scan whose first
stage barrier in one warp can never complete (mpm_test_inject(1): the
barrier expects 16 bytes more than its copy brings).  The warp's bounded
wait gives up, it records MPM_ETIMEOUT, drains its own copies and returns;
the search reports MPM_ETIMEOUT and the same handle then searches exactly."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_1405_5483_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def mpm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1405_5483_gb300 import build_lib
    build_lib.build()
    import paper_1405_5483_gb300 as mpm
    return mpm


@pytest.fixture(scope="module")
def native():
    from oracle import native
    native.build()
    return native


def as_u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("kernel", [2, 3])
def test_bounded_wait_runs_out_and_the_handle_recovers(mpm, native, kernel):
    from paper_1405_5483_gb300._native import MPM_ETIMEOUT
    case = W.protein_case(1 << 26, 200, 32, 100, cfg=21)   # 64 MiB: rows through TMA
    T = torch.from_numpy(case.T).cuda()
    m = mpm.Matcher(case.P, sigma=20, q=3, sigma_r=16, k=1, map_kind=2, kernel=kernel)
    want = native.aho_corasick(case.T, case.P, threads=8)
    pos, pid = m.search(T)
    assert np.array_equal(as_u32(pos), want[0])
    assert m.stats["specialised"] == 1
    assert mpm.lib().mpm_test_inject(1) == 0
    t0 = time.time()
    with pytest.raises(mpm.MpmError) as e:
        m.search(T)
    assert e.value.code == MPM_ETIMEOUT
    assert time.time() - t0 < 60
    # the hook is one-shot, and the handle's next searches are exact
    for _ in range(2):
        pos, pid = m.search(T)
        assert np.array_equal(as_u32(pos), want[0]) and np.array_equal(as_u32(pid), want[1])


def test_inject_rejects_unknown_faults(mpm):
    assert mpm.lib().mpm_test_inject(7) == mpm.MPM_EINVAL
    assert mpm.lib().mpm_test_inject(0) == 0

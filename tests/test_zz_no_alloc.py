"""mpm_search_noalloc: a search that allocates no device memory.

Some callers cannot let a library call cudaMalloc while they search: a
program whose device memory is all handed out by its own pool or caching
allocator (an extra cudaMalloc can fail or fragment that pool), or a
latency-sensitive server in which cudaMalloc and cudaFree may synchronise
the device and stall other streams.  mpm_search_noalloc serves them by
keeping its scratch in a fixed device array inside the library.

These tests call it through the C ABI and require its occurrence lists to be
identical (integers, so no tolerance) to those of mpm_search, on two calls
in a row with different texts, so that anything the shared array keeps from
the previous call would show.  The file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mpm():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1405_5483_gb300 import build_lib
    build_lib.build()
    import paper_1405_5483_gb300 as mpm
    return mpm


def _noalloc(mpm, matcher, T, cap):
    out_pos = torch.full((cap,), -1, dtype=torch.int32, device=T.device)
    out_pid = torch.full((cap,), -1, dtype=torch.int32, device=T.device)
    z = ctypes.c_size_t(cap)
    lib = mpm.lib()
    lib.mpm_set_stream(matcher._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    rc = lib.mpm_search_noalloc(matcher._h, T.data_ptr(), T.numel(), out_pos.data_ptr(),
                                out_pid.data_ptr(), ctypes.byref(z))
    torch.cuda.synchronize()
    return rc, z.value, out_pos, out_pid


def test_noalloc_equals_search_on_two_calls_in_a_row(mpm):
    from paper_1405_5483_gb300 import workloads as W
    cases = [W.dna_case(1 << 20, 100, 16, 50), W.protein_case((1 << 22) + 13, 300, 32, 150)]
    built = []
    for c in cases:
        m = mpm.Matcher(c.P, sigma=c.sigma)
        T = torch.from_numpy(c.T).cuda()
        ref_pos, ref_pid = m.search(T)
        torch.cuda.synchronize()
        built.append((m, T, ref_pos.cpu().numpy(), ref_pid.cpu().numpy()))
    for rep in range(2):
        for m, T, ref_pos, ref_pid in built:
            rc, z, pos, pid = _noalloc(mpm, m, T, 4096)
            assert rc == mpm.MPM_OK, mpm.lib().mpm_strerror(rc)
            assert z == ref_pos.size
            assert np.array_equal(pos[:z].cpu().numpy(), ref_pos)
            assert np.array_equal(pid[:z].cpu().numpy(), ref_pid)
            assert m.stats["z"] == z


def test_noalloc_rejects_more_occurrences_than_its_scratch_holds(mpm):
    from paper_1405_5483_gb300._native import MPM_ESCRATCH, NOALLOC_MAX_OCCURRENCES
    T = torch.full((NOALLOC_MAX_OCCURRENCES * 2,), 65, dtype=torch.uint8, device="cuda")
    P = np.full((1, 8), 65, np.uint8)
    m = mpm.Matcher(P, sigma=2)
    rc, z, _, _ = _noalloc(mpm, m, T, 1 << 16)
    assert rc == MPM_ESCRATCH
    assert z == T.numel() - 8 + 1
    # the regular search still handles it
    pos, _ = m.search(T)
    assert pos.numel() == z

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


# The automatic choice (the specialised scan that verifies its candidates
# itself), the generic kernel and the split specialised scan: the last two
# keep candidate records in the shared array and verify them in a second
# kernel.
KERNELS = [("auto", {}), ("generic", {"kernel": 1}), ("split", {"kernel": 3})]


@pytest.mark.parametrize("name,kw", KERNELS, ids=[k for k, _ in KERNELS])
def test_noalloc_equals_search_on_two_calls_in_a_row(mpm, name, kw):
    from paper_1405_5483_gb300 import workloads as W
    cases = [W.dna_case(1 << 20, 100, 16, 50), W.protein_case((1 << 22) + 13, 300, 32, 150)]
    built = []
    for c in cases:
        m = mpm.Matcher(c.P, sigma=c.sigma, **kw)
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


def test_noalloc_rejects_more_candidates_than_its_scratch_holds(mpm):
    from paper_1405_5483_gb300._native import MPM_ESCRATCH, NOALLOC_MAX_CANDIDATES
    # every q-gram of an all-A text matches the filter of AAAAAAAAAAAAAAAC
    # (q = 2: seven positions, each accepting "AA"), so every sampled q-gram
    # is a candidate record while no window is an occurrence
    n = 4 * NOALLOC_MAX_CANDIDATES
    T = torch.full((n,), 65, dtype=torch.uint8, device="cuda")
    P = np.frombuffer(b"AAAAAAAAAAAAAAAC", np.uint8).reshape(1, 16)
    for kernel in (1, 3):
        m = mpm.Matcher(P, sigma=4, q=2, k=1, sigma_r=4, map_kind=mpm.MAP_RANK, kernel=kernel)
        rc, z, _, _ = _noalloc(mpm, m, T, 4096)
        assert rc == MPM_ESCRATCH
        assert z == 0
        assert m.stats["candidates"] > NOALLOC_MAX_CANDIDATES
        # the regular search finds the same (empty) list
        pos, _ = m.search(T)
        assert pos.numel() == 0


def test_noalloc_after_pipelined_search_into_the_same_outputs(mpm):
    """A pipelined search's closing sort runs on a side stream; a following
    allocation-free search into the same outputs is ordered after it."""
    from paper_1405_5483_gb300 import workloads as W
    c = W.protein_case(1 << 24, 1000, 32, 500)
    m = mpm.Matcher(c.P, sigma=c.sigma)
    T1 = torch.from_numpy(c.T).cuda()
    # the first quarter of the text: a different, shorter occurrence list
    T2 = T1[: 1 << 22].clone()
    ref_pos, ref_pid = m.search(T2)
    ref_pos, ref_pid = ref_pos.cpu().numpy(), ref_pid.cpu().numpy()
    cap = 4096
    out_pos = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    out_pid = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    lib = mpm.lib()
    for _ in range(3):
        m.search_async(T1, out_pos, out_pid, status)
        z = ctypes.c_size_t(cap)
        rc = lib.mpm_search_noalloc(m._h, T2.data_ptr(), T2.numel(), out_pos.data_ptr(),
                                    out_pid.data_ptr(), ctypes.byref(z))
        assert rc == mpm.MPM_OK, lib.mpm_strerror(rc)
        m.sync()
        zz = z.value
        assert zz == ref_pos.size
        assert np.array_equal(out_pos[:zz].cpu().numpy(), ref_pos)
        assert np.array_equal(out_pid[:zz].cpu().numpy(), ref_pid)

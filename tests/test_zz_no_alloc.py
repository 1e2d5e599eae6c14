"""msc_compress_noalloc: path compression for callers that cannot allocate
device memory (processes whose device memory belongs to another allocator or
a fixed budget, code that must not risk the synchronisation allocation can
cause).  It keeps its scratch in a static device array instead of a caller
workspace.

Checked through the C ABI against msc_compress (the workspace entry point),
bit for bit, on two calls in a row with different sizes and data -- the
second call must not see anything the first left in the shared array -- and
against the oracle's memoised walk to each vertex's root.  A call at the
maximum size leaves the device's free memory unchanged.
This file is collected last so that a run stopping at the first failure has
run every other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def chains(n, seed, roots, span):
    """Parent pointers of a random forest: vertex perm[i] points at one of the
    `span` vertices before it, so paths are long (~n / (roots * span))."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n).astype(np.int64)
    ptr = np.empty(n, np.int32)
    i = np.arange(n, dtype=np.int64)
    back = 1 + rng.integers(0, span, n) % np.maximum(i, 1)
    parent = np.where(i < roots, perm, perm[np.maximum(i - back, 0)])
    ptr[perm] = parent
    return ptr


@pytest.fixture(scope="module")
def m():
    import paper_2409_03771_gb300 as msc
    from paper_2409_03771_gb300 import _build

    _build.build()
    msc.load()
    return msc


def run_both(m, ptr_host):
    n = ptr_host.size
    ref = torch.from_numpy(ptr_host).cuda()
    got = ref.clone()
    st_ref = torch.zeros(1, dtype=torch.int32, device="cuda")
    st_got = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    ws = torch.empty(m.msc_workspace_bytes(m.OP_COMPRESS, n), dtype=torch.uint8, device="cuda")
    assert m.msc_compress(ref, n, ws, ws.numel(), st_ref) == m.OK
    assert m.msc_compress_noalloc(got, n, st_got) == m.OK
    torch.cuda.synchronize()
    assert int(st_ref.item()) == m.OK and int(st_got.item()) == m.OK
    return ref, got


def test_noalloc_matches_workspace_entry_on_two_calls_in_a_row(m, oracle_mod):
    first = chains(m.NOALLOC_MAX_N, seed=1, roots=3, span=2)  # maximum size, long paths
    second = chains(1_000_003, seed=2, roots=50, span=7)  # smaller, different data
    for host in (first, second):
        ref, got = run_both(m, host)
        assert torch.equal(ref, got)
        # every entry is its vertex's root, as the oracle's walk finds it
        np.testing.assert_array_equal(got.cpu().numpy(), oracle_mod.walk_memo(host))


def test_noalloc_leaves_free_device_memory_unchanged(m):
    host = chains(m.NOALLOC_MAX_N, seed=3, roots=5, span=3)
    ptr = torch.from_numpy(host).cuda()
    warm = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert m.msc_compress_noalloc(warm, 1, st) == m.OK  # warm-up: loads the device code
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    assert m.msc_compress_noalloc(ptr, ptr.numel(), st) == m.OK
    torch.cuda.synchronize()
    assert int(st.item()) == m.OK
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_rejects_sizes_beyond_its_scratch(m):
    n = m.NOALLOC_MAX_N + 1
    ptr = torch.arange(n, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert m.msc_compress_noalloc(ptr, n, st) == m.ERR_TOO_LARGE
    assert "exceeds a limit" in m.msc_status_string(m.ERR_TOO_LARGE)
    # device-side errors still reach the status word
    cyc = torch.tensor([1, 2, 0], dtype=torch.int32, device="cuda")
    assert m.msc_compress_noalloc(cyc, 3, st) == m.OK
    torch.cuda.synchronize()
    assert int(st.item()) == m.ERR_NOT_CONVERGED

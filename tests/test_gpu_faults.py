"""Failure paths on the GPU without faulting it: a bounded device wait that
runs out (a flag nothing sets) is reported as FASTID_ETIMEOUT and leaves the
context usable; an allocation the device cannot satisfy is FASTID_ENOMEM with
nothing enqueued."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1707_00516_gb300 import binding as B  # noqa: E402
from paper_1707_00516_gb300.search import Searcher, words64  # noqa: E402


@pytest.fixture(scope="module")
def s():
    import __graft_entry__
    __graft_entry__.build()
    sr = Searcher(0, B.FORM_TENSOR)
    yield sr
    sr.ctx.close()


def _small_topk(s):
    rng = np.random.default_rng(5)
    R = (rng.random((500, 300)) < 0.3).astype(np.uint8)
    Q = (rng.random((20, 300)) < 0.3).astype(np.uint8)
    modes = (rng.random(20) < 0.5).astype(np.uint8)
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), 300)
    q = torch.empty((20, words64(300)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(Q).cuda(), 300, q)
    sc, ix = s.topk(db, q, torch.from_numpy(modes).cuda(), 8)
    mis, une = oracle.scores(R, Q)
    es, ei = oracle.topk(oracle.select(mis, une, modes), 8, B.NO_THRESHOLD)
    ok = np.array_equal(sc.cpu().numpy().view(np.uint32), es) and np.array_equal(ix.cpu().numpy(), ei)
    db.close()
    return ok


def test_bounded_wait_times_out_and_context_survives(s):
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.fastid_wait_flag(s.ctx, flag, 100)  # nothing sets the flag
    assert B.fastid_sync_status(s.ctx) == B.ETIMEOUT
    # the status word was read and cleared; the context still computes
    assert _small_topk(s)
    assert B.fastid_sync_status(s.ctx) == B.OK


def test_bounded_wait_ends_when_flag_set(s):
    flag = torch.ones(1, dtype=torch.int32, device="cuda")
    B.fastid_wait_flag(s.ctx, flag, 5000)
    assert B.fastid_sync_status(s.ctx) == B.OK


def test_wait_flag_arguments(s):
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    for ms in (0, 10001):
        with pytest.raises(B.FastIDError) as e:
            B.fastid_wait_flag(s.ctx, flag, ms)
        assert e.value.status == B.EINVAL


def test_allocation_failure_is_enomem(s):
    """A database far larger than the device (2^31 - 1 references x 65536 loci,
    ~17.6 TB packed): the allocation fails, the call returns FASTID_ENOMEM and
    the caller's buffer is never read."""
    small = torch.zeros((4, 1024), dtype=torch.int64, device="cuda")
    lib = B.load_library()
    import ctypes
    out = ctypes.c_void_p()
    st = lib.fastid_load_refs(s.ctx.handle, small.data_ptr(), (1 << 31) - 1, 65536, 1024, 0, ctypes.byref(out), None)
    assert st == B.ENOMEM
    assert not out.value
    assert _small_topk(s)
    assert B.fastid_sync_status(s.ctx) == B.OK


def test_database_file_roundtrip(s, tmp_path):
    """fastid_save_refs then fastid_load_refs_file: the reloaded database (with
    and without its FP8 copy) gives the same top-k as the original; a damaged
    or truncated file is FASTID_EINVAL."""
    rng = np.random.default_rng(8)
    n_loci = 777
    R = (rng.random((2500, n_loci)) < 0.3).astype(np.uint8)
    Q = (rng.random((40, n_loci)) < 0.3).astype(np.uint8)
    modes = (rng.random(40) < 0.5).astype(np.uint8)
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci)
    path = str(tmp_path / "refs.fastiddb")
    B.fastid_save_refs(s.ctx, db, path)
    q = torch.empty((40, words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(Q).cuda(), n_loci, q)
    m = torch.from_numpy(modes).cuda()
    sc0, ix0 = s.topk(db, q, m, 9)
    for flags in (B.REFS_TENSOR, 0):
        db2 = B.fastid_load_refs_file(s.ctx, path, flags)
        assert db2.n_refs == 2500 and db2.n_loci == n_loci and db2.info()["flags"] == flags
        sc1, ix1 = s.topk(db2, q, m, 9)
        assert torch.equal(sc0, sc1) and torch.equal(ix0, ix1)
        db2.close()
    db.close()
    raw = open(path, "rb").read()
    bad = tmp_path / "bad.fastiddb"
    bad.write_bytes(b"NOTADB!!" + raw[8:])
    with pytest.raises(B.FastIDError) as e:
        B.fastid_load_refs_file(s.ctx, str(bad), 0)
    assert e.value.status == B.EINVAL
    bad.write_bytes(raw[: len(raw) // 2])
    with pytest.raises(B.FastIDError) as e:
        B.fastid_load_refs_file(s.ctx, str(bad), 0)
    assert e.value.status == B.EINVAL
    assert B.fastid_sync_status(s.ctx) == B.OK


def test_search_host_raises_on_device_condition(s):
    """The host-buffer path reads the status word before returning: with a
    planted timeout (a bounded wait on a flag nothing sets) search_host raises
    FASTID_ETIMEOUT instead of returning results; the next call returns the
    oracle's lists."""
    rng = np.random.default_rng(9)
    R = (rng.random((700, 200)) < 0.3).astype(np.uint8)
    src = (rng.random((30, 200)) < 0.3).astype(np.uint8)
    off = np.arange(31, dtype=np.int32)  # one contributor per query
    modes = (rng.random(30) < 0.5).astype(np.uint8)
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), 200)
    B.fastid_wait_flag(s.ctx, torch.zeros(1, dtype=torch.int32, device="cuda"), 50)
    with pytest.raises(B.FastIDError) as e:
        s.search_host(db, src, off, modes, 6)
    assert e.value.status == B.ETIMEOUT
    sc, ix, _, _ = s.search_host(db, src, off, modes, 6)
    mis, une = oracle.scores(R, src)
    es, ei = oracle.topk(oracle.select(mis, une, modes), 6)
    assert np.array_equal(sc, es) and np.array_equal(ix, ei)
    db.close()
    assert B.fastid_sync_status(s.ctx) == B.OK

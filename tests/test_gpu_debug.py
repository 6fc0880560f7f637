"""The FASTID_DEBUG build on the GPU: with its device-side consistency checks
(the merge reads only slots inside the schedule) and its host-side schedule
self-check, the tensor form (paired FP8 and packed rows, both with a schedule
tail) and a two-panel batched plan give the oracle's lists, and the status
word stays clear.  It runs in a subprocess that loads only the debug
library."""
import os
import subprocess
import sys

import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import numpy as np, torch
from paper_1707_00516_gb300 import build as Bd
from paper_1707_00516_gb300 import binding as B
B.load_library(Bd.build(debug=True))
import gen, oracle
from paper_1707_00516_gb300.search import Searcher, words64

def check(s, what):
    st = B.fastid_sync_status(s.ctx)
    assert st == B.OK, (what, st)

# 2048 queries (8 tile pairs) x 25,600 references: an 8 x 9 grid plus a tail
n_refs, n_loci, n_q, k = 25_600, 96, 2048, 16
rng = np.random.default_rng(77)
thr = gen.maf_thresholds(77, n_loci)
R = gen.allele_rows(77, gen.STREAM_DB, np.arange(n_refs), thr)
Q = (rng.random((n_q, n_loci)) < 0.35).astype(np.uint8)
Q[:32] = R[rng.integers(0, n_refs, 32)]
modes = (rng.random(n_q) < 0.5).astype(np.uint8)
mis, une = oracle.scores(R, Q)
es, ei = oracle.topk(oracle.select(mis, une, modes), k)
for form in (B.FORM_TENSOR, B.FORM_TENSOR_PACKED, B.FORM_TENSOR_FP4, B.FORM_TENSOR_FP4_PACKED, B.FORM_PLAIN):
    s = Searcher(0, form)
    db = s.load_refs_alleles(torch.from_numpy(R).cuda(), n_loci)
    q = torch.empty((n_q, words64(n_loci)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(Q).cuda(), n_loci, q)
    sc, ix = s.topk(db, q, torch.from_numpy(modes).cuda(), k)
    torch.cuda.synchronize()
    check(s, form)
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), es), form
    assert np.array_equal(ix.cpu().numpy(), ei), form
    db.close(); s.ctx.close()

# a two-panel plan, batches of uneven size
s = Searcher(0, B.FORM_TENSOR)
panels = [(3000, 300), (5000, 1100)]
dbs, Rs = [], []
for i, (nr, nl) in enumerate(panels):
    t = gen.maf_thresholds(90 + i, nl)
    Rp = gen.allele_rows(90 + i, gen.STREAM_DB, np.arange(nr), t)
    Rs.append(Rp)
    dbs.append(s.load_refs_alleles(torch.from_numpy(Rp).cuda(), nl, flags=B.REFS_TENSOR))
sizes, pidx = [5, 300, 129, 1, 260], [0, 1, 0, 1, 1]
batches, expect = [], []
for b, (n, p) in enumerate(zip(sizes, pidx)):
    nl = panels[p][1]
    Qb = (rng.random((n, nl)) < 0.3).astype(np.uint8)
    mb = (rng.random(n) < 0.5).astype(np.uint8)
    qd = torch.empty((n, words64(nl)), dtype=torch.int64, device="cuda")
    B.fastid_pack(s.ctx, torch.from_numpy(Qb).cuda(), nl, qd)
    batches.append((p, qd, torch.from_numpy(mb).cuda(), torch.zeros((n, 12), dtype=torch.int32, device="cuda"),
                    torch.zeros((n, 12), dtype=torch.int64, device="cuda")))
    m1, u1 = oracle.scores(Rs[p], Qb)
    expect.append(oracle.topk(oracle.select(m1, u1, mb), 12))
plan = B.Plan(s.ctx, dbs, batches, 12, B.NO_THRESHOLD, B.VARIANT_TENSOR_PAIR)
plan.run()
torch.cuda.synchronize()
check(s, "plan")
for (p, qd, md, sc, ix), (es2, ei2) in zip(batches, expect):
    assert np.array_equal(sc.cpu().numpy().view(np.uint32), es2)
    assert np.array_equal(ix.cpu().numpy(), ei2)
plan.close()
for d in dbs:
    d.close()
s.ctx.close()
print("DEBUG BUILD OK")
"""


def test_debug_build_parity():
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCRIPT], capture_output=True, text=True,
                       timeout=1200, cwd=ROOT)
    assert r.returncode == 0 and "DEBUG BUILD OK" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])

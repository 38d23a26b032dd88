"""Host logic of the persistent tuning table (no GPU: a stand-in problem records calls)."""
from paper_1909_03948_gb300 import tuning


class FakeProblem:
    dim, N = 2, 64

    def __init__(self):
        self.applied = None
        self.autotuned = 0

    def set_tuning(self, **kw):
        self.applied = kw

    def autotune(self, nrhs, X=None):
        self.autotuned += 1
        self.block = X
        return {"nu": 1, "omega": 0.8, "col_chunk": 0, "max_blocks": 4096}, 1.5


def test_autotune_once_then_reuse(tmp_path):
    path = str(tmp_path / "t.json")
    p = FakeProblem()
    s, ms, src = tuning.tuned(p, 40, path=path)
    assert src == "autotune" and p.autotuned == 1 and ms == 1.5
    q = FakeProblem()
    s2, ms2, src2 = tuning.tuned(q, 40, path=path)
    assert src2 == "table" and q.autotuned == 0 and q.applied == s
    # other block widths and sizes are separate entries
    s3, _, src3 = tuning.tuned(q, 8, path=path)
    assert src3 == "autotune" and q.block is None
    assert len(tuning.load(path)) == 2
    # the caller's block, when given, is what the autotuner times
    r = FakeProblem()
    blk = object()
    tuning.tuned(r, 12, path=path, X=blk)
    assert r.autotuned == 1 and r.block is blk

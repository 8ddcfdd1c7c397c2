"""Host-side logic that needs no GPU, with fakes in place of the library's
GPU calls: the batched autotuner's choice and its cache, and the
convergence study's bookkeeping and statistics."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


class _FakeBatched:
    """Stands in for prcg_batched_*: configurations cost a fixed time each;
    some cannot be configured."""

    def __init__(self, binding, times, refuse=()):
        self.binding, self.times, self.refuse = binding, times, set(refuse)
        self.cfg = None
        self.solves = 0

    def configure(self, bt, cluster, threads):
        if (cluster, threads) in self.refuse:
            raise self.binding.PrcgError(self.binding.PRCG_ERR_UNSUPPORTED, "not resident")
        self.cfg = (cluster, threads)

    def configure_split(self, bt, nbig, cb, tb, cr, tr):
        key = (nbig, cb, tb, cr, tr)
        if key in self.refuse or key not in self.times:
            raise self.binding.PrcgError(self.binding.PRCG_ERR_INVALID, "no such split")
        self.cfg = key

    def solve(self, bt, b, x, tol, maxit, *args):
        self.solves += 1
        x.fill_(1.0)
        return 0

    def last_ms(self, bt):
        return self.times[self.cfg]


def _install(monkeypatch, autotune, fake):
    monkeypatch.setattr(autotune.binding, "prcg_batched_configure", fake.configure)
    monkeypatch.setattr(autotune.binding, "prcg_batched_configure_split", fake.configure_split)
    monkeypatch.setattr(autotune.binding, "prcg_batched_solve", fake.solve)
    monkeypatch.setattr(autotune.binding, "prcg_batched_last_ms", fake.last_ms)


def test_tuner_picks_fastest_skips_unlaunchable_and_caches(G, monkeypatch, tmp_path):
    import torch
    from paper_1905_01549_gb300 import autotune
    cands = [(1, 256), (2, 512), (8, 512), (16, 256)]
    times = {(1, 256): 9.0, (2, 512): 4.0, (8, 512): 2.5, (16, 256): 1.0}
    fake = _FakeBatched(autotune.binding, times, refuse={(16, 256)})
    _install(monkeypatch, autotune, fake)
    cache = str(tmp_path / "tune.json")
    x0 = torch.zeros(10, dtype=torch.float64)
    key = autotune.batch_key([32, 48], [40, 64], [0.0, 0.05], 0, 1e-8, "dev")
    c, t, ms, table = autotune.tune(None, None, x0, 1e-8, 100, key=key, candidates=cands,
                                    cache_path=cache)
    assert (c, t, ms) == (8, 512, 2.5) and fake.cfg == (8, 512)
    assert (16, 256, None) in [tuple(r) for r in table]     # refused, recorded, skipped
    assert bool((x0 == 0).all())                             # x0 is left unchanged
    n_solves = fake.solves
    fake.cfg = None
    c2, t2, ms2, _ = autotune.tune(None, None, x0, 1e-8, 100, key=key, candidates=cands,
                                   cache_path=cache)
    assert (c2, t2, ms2) == (8, 512, 2.5) and fake.cfg == (8, 512)
    assert fake.solves == n_solves                           # answered from the cache


def test_tuner_picks_and_caches_a_split_launch(G, monkeypatch, tmp_path):
    import torch
    from paper_1905_01549_gb300 import autotune
    cands = [(8, 512), (16, 512)]
    splits = [(4, 16, 512, 8, 512), (8, 16, 512, 8, 512), (600, 16, 512, 8, 512)]
    times = {(8, 512): 3.0, (16, 512): 4.0, (4, 16, 512, 8, 512): 2.0,
             (8, 16, 512, 8, 512): 2.4}
    fake = _FakeBatched(autotune.binding, times)
    _install(monkeypatch, autotune, fake)
    cache = str(tmp_path / "tune.json")
    x0 = torch.zeros(10, dtype=torch.float64)
    key = autotune.batch_key([32, 448], [40, 448], [0.0, 0.05], 0, 1e-8, "dev")
    c, t, ms, table = autotune.tune(None, None, x0, 1e-8, 100, key=key, candidates=cands,
                                    splits=splits, cache_path=cache)
    assert (c, t, ms) == (16, 512, 2.0) and fake.cfg == (4, 16, 512, 8, 512)
    assert (600, 16, 512, 8, 512, None) in [tuple(r) for r in table]   # rejected: recorded
    n_solves = fake.solves
    fake.cfg = None
    autotune.tune(None, None, x0, 1e-8, 100, key=key, candidates=cands, splits=splits,
                  cache_path=cache)
    assert fake.cfg == (4, 16, 512, 8, 512) and fake.solves == n_solves   # split re-applied


def test_tuner_fails_loudly_when_nothing_launches(G, monkeypatch, tmp_path):
    import torch
    from paper_1905_01549_gb300 import autotune
    fake = _FakeBatched(autotune.binding, {}, refuse={(1, 256), (2, 256)})
    _install(monkeypatch, autotune, fake)
    with pytest.raises(RuntimeError):
        autotune.tune(None, None, torch.zeros(4, dtype=torch.float64), 1e-8, 10,
                      candidates=[(1, 256), (2, 256)], splits=[(2, 16, 512, 8, 512)],
                      cache_path=str(tmp_path / "t.json"))


def test_tuning_key_separates_what_changes_the_choice(G):
    from paper_1905_01549_gb300 import autotune
    base = ([32, 48], [40, 64], [0.0, 0.05], 0, 1e-8, "GB300")
    k = autotune.batch_key(*base)
    assert k == autotune.batch_key(*base)
    variants = [([32, 49], [40, 64], [0.0, 0.05], 0, 1e-8, "GB300"),
                ([32, 48], [40, 64], [0.0, 0.06], 0, 1e-8, "GB300"),
                ([32, 48], [40, 64], [0.0, 0.05], 1, 1e-8, "GB300"),
                ([32, 48], [40, 64], [0.0, 0.05], 0, 1e-6, "GB300"),
                ([32, 48], [40, 64], [0.0, 0.05], 0, 1e-8, "other GPU")]
    assert len({autotune.batch_key(*v) for v in variants} | {k}) == 6


def test_error_curve_statistics(G):
    from paper_1905_01549_gb300.convergence import ErrorCurve
    c = ErrorCurve(np.arange(6), np.array([1.0, 1e-2, 2e-5, 9e-6, 1e-9, 3e-9]), None)
    assert c.iterations_to(1e5) == 3 and c.iterations_to(1e10) is None
    assert math.isclose(c.min_log10(), -9.0)


class _FakeSolver:
    """x_k = x* (1 - 2^-k), A = I; breaks down at k = 7."""

    def __init__(self, n):
        import torch
        self.n = n
        self.xs = torch.ones(n, dtype=torch.float64)

    def error_anorm(self, xs, x):
        return float(((xs - x) ** 2).sum().sqrt())

    def solve(self, b, x0, variant, tol, maxit):
        from types import SimpleNamespace
        k = min(maxit, 7)
        x0.copy_(self.xs * (1.0 - 0.5 ** k))
        status = 2 if maxit >= 7 else 1
        return SimpleNamespace(iters=k, status=status)


def test_error_curve_reruns_and_stops_at_breakdown(G):
    import torch
    from paper_1905_01549_gb300 import convergence
    S = _FakeSolver(5)
    curve = convergence.error_curve(S, None, S.xs, "pr", kmax=20,
                                    x0=torch.zeros(5, dtype=torch.float64))
    assert list(curve.k) == list(range(8)) and curve.breakdown_at == 7
    assert np.allclose(curve.err, 0.5 ** np.arange(8))
    assert curve.iterations_to(100) == 7 and math.isclose(curve.min_log10(), 7 * math.log10(0.5))

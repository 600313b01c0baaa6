"""Host logic of the Section 5.2 searches (no device): the candidate order and
stopping rule of minimal_shift, the damping lists damping_search hands to the
solver, and the argmin of lfa_damping, with the library's factor calls
replaced by scripted fakes.  Invalid LFA arguments are refused by the C ABI
before any device work."""
import numpy as np
import pytest

from paper_2511_16808_gb300 import hz, tuning


def test_minimal_shift_tries_increasing_and_stops(monkeypatch):
    seen = []
    factors = {0.0: 1.7, 0.05: 1.4, 0.1: 1.05, 0.2: 0.6, 0.3: 0.4}

    def fake(dim, n, kappa, omega, gamma, alpha, levels, seed, cf_max_iter, **opts):
        seen.append(alpha)
        assert cf_max_iter == 60 and opts == {"patch": "plus"}
        return factors[alpha], 60
    monkeypatch.setattr(tuning, "_factor_for", fake)
    a, table = tuning.minimal_shift(2, 65, None, 1.0, None, 3, [0.3, 0.1, 0.0, 0.2, 0.05], patch="plus")
    assert a == 0.2 and seen == [0.0, 0.05, 0.1, 0.2]
    assert [t[0] for t in table] == seen


def test_minimal_shift_none_when_all_diverge(monkeypatch):
    monkeypatch.setattr(tuning, "_factor_for", lambda *a, **k: (1.2, 60))
    a, table = tuning.minimal_shift(2, 65, None, 1.0, None, 3, [0.1, 0.2])
    assert a is None and len(table) == 2


def test_damping_search_fixes_finer_levels(monkeypatch):
    calls = []

    def fake(dim, n, kappa, omega, gamma, alpha, levels, seed, cf_max_iter, **opts):
        d = list(opts["damping"])
        calls.append(d)
        return abs(d[1] - 0.55) + 0.1, 10          # best at w = 0.55 on level 1
    monkeypatch.setattr(tuning, "_factor_for", fake)
    best, table = tuning.damping_search(2, 65, None, 1.0, None, 0.2, 4, 1, [0.4, 0.55, 0.7], fixed=(0.81,),
                                        patch="rb")
    assert best == 0.55 and [w for w, _ in table] == [0.4, 0.55, 0.7]
    for d, w in zip(calls, [0.4, 0.55, 0.7]):
        assert d[0] == 0.81 and d[1] == w
        # coarser levels keep the paper's table for the RB patch
        assert d[2] == hz.hz_default_damping(2, "rb", 2) and d[3] == hz.hz_default_damping(2, "rb", 3)


def test_lfa_damping_argmin(monkeypatch):
    ws = np.array([0.5, 0.7, 0.9])
    monkeypatch.setattr(hz, "hz_lfa_factors",
                        lambda *a, **k: (np.array([0.9, 0.6, 0.7]), np.array([0.5, np.nan, 0.4])))
    best, mu, rho = tuning.lfa_damping(2, {}, "rb", ws)
    assert best == 0.9                               # NaN (no converged eigenvalue) is never chosen
    best_mu, _, _ = tuning.lfa_damping(2, {}, "rb", ws, by="mu")
    assert best_mu == 0.7


@pytest.mark.parametrize("kw", [dict(nw_zero=True), dict(samples=1), dict(rk="mixed"), dict(nu=(9, 8))])
def test_lfa_arguments_refused(kw):
    st = {(0, 0): 4.0, (1, 0): -1.0, (-1, 0): -1.0, (0, 1): -1.0, (0, -1): -1.0}
    ws = [] if kw.get("nw_zero") else [0.8]
    with pytest.raises(hz.HzError) as e:
        hz.hz_lfa_factors(2, st, "plus", ws, kw.get("rk", "cubic"), "cubic", *kw.get("nu", (1, 1)),
                          samples=kw.get("samples", 16))
    assert e.value.status == 1                       # HZ_ERR_INVALID_ARG

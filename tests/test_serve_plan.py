"""CPU tests of the server's packing rule, fe_serve_plan (host-only code in
the library; no device is touched)."""
import numpy as np
import pytest

from paper_0704_2344_gb300 import fe as fe_mod


@pytest.fixture(scope="module")
def fe():
    try:
        fe_mod.load()
    except FileNotFoundError:
        from paper_0704_2344_gb300 import build
        build.build()
    return fe_mod


def _demand(rows, width, cap, work):
    r = max(rows, 1)
    return max(1, min(-(-r * width // work), r, cap))


def test_plan_examples(fe):
    taken, n = fe.fe_serve_plan([125000, 500, 300], [16, 16, 16], 152, 2048)
    assert taken == 1 and list(n) == [152, 0, 0]
    taken, n = fe.fe_serve_plan([500, 8000, 125000, 300], [4, 8, 4, 4], 152, 2048)
    # the width-8 request waits; the big width-4 request does not fit next to the first
    assert taken == 2 and n[1] == 0 and n[2] == 0 and n[0] >= 1 and n[3] >= 1
    taken, n = fe.fe_serve_plan([20000, 8000, 3000], [8, 8, 8], 152, 2048)
    assert taken == 3 and n.sum() == 152 and n[0] >= 79 and n[1] >= 32 and n[2] >= 12
    assert fe.fe_serve_plan([], [], 152, 2048)[0] == 0
    # a per-request cap lets two large requests share the device
    taken, n = fe.fe_serve_plan([125000, 125000, 500], [16, 16, 16], 152, 2048, max_job_ctas=76)
    assert taken == 2 and list(n) == [76, 76, 0]


@pytest.mark.parametrize("seed", range(40))
def test_plan_invariants(fe, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    rows = np.exp(rng.uniform(np.log(1), np.log(200000), n)).astype(np.int64)
    widths = 2 ** rng.integers(0, 6, n)
    max_ctas = int(rng.integers(1, 200))
    work = int(rng.choice([256, 1024, 2048, 8192]))
    job_cap = int(rng.choice([0, max(1, max_ctas // 2), max_ctas]))
    cap = job_cap if 1 <= job_cap <= max_ctas else max_ctas
    taken, cta = fe.fe_serve_plan(rows, widths, max_ctas, work, max_job_ctas=job_cap)
    sel = cta > 0
    assert taken == sel.sum() >= 1
    assert sel[0]                                   # the oldest request is always taken
    assert cta.sum() <= max_ctas
    assert np.all(widths[sel] == widths[0])         # one tile width per launch
    assert np.all(cta[sel] <= np.maximum(rows[sel], 1)) and np.all(cta[sel] <= cap)
    for i in np.flatnonzero(sel):
        if i == 0:
            assert cta[0] >= min(_demand(rows[0], widths[0], cap, work), max_ctas)
        else:
            assert cta[i] >= _demand(rows[i], widths[i], cap, work)
    # a same-width request left out did not fit in what the earlier ones left
    used = 0
    for i in range(n):
        if widths[i] != widths[0]:
            continue
        d = _demand(rows[i], widths[i], cap, work)
        if i == 0:
            used += min(d, max_ctas)
        elif d <= max_ctas - used:
            assert sel[i]
            used += d
        else:
            assert not sel[i]

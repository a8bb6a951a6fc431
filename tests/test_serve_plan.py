"""CPU tests of the server's scheduling rule, fe_serve_plan (host-only code
in the library; no device is touched)."""
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
    # one large request takes the whole device; the others wait
    taken, n = fe.fe_serve_plan([125000, 500, 300], [16, 16, 16], 152, 2048)
    assert taken == 1 and list(n) == [152, 0, 0]
    # widths mix in one segment; a later, smaller request backfills
    taken, n = fe.fe_serve_plan([500, 8000, 125000, 300], [4, 8, 4, 4], 152, 2048)
    assert list(n) == [1, 32, 0, 1] and taken == 3
    # counts never grow to fill the device
    taken, n = fe.fe_serve_plan([20000, 8000, 3000], [8, 8, 8], 152, 2048)
    assert taken == 3 and list(n) == [79, 32, 12]
    assert fe.fe_serve_plan([], [], 152, 2048)[0] == 0
    # a per-request cap lets two large requests share the device
    taken, n = fe.fe_serve_plan([125000, 125000, 500], [16, 16, 16], 152, 2048, max_job_ctas=76)
    assert taken == 2 and list(n) == [76, 76, 0]


def test_plan_count_does_not_depend_on_the_mix(fe):
    """A request's CTA count is the same alone, behind others or among others
    (only whether it runs in this segment depends on them)."""
    alone = fe.fe_serve_plan([8000], [4], 152, 1024)[1][0]
    for rows, widths in (([8000, 500, 40000], [4, 1, 16]), ([300, 8000], [2, 4]), ([50, 50, 8000, 7], [1, 1, 4, 32])):
        i = rows.index(8000)
        _, n = fe.fe_serve_plan(rows, widths, 152, 1024)
        assert n[i] in (0, alone)


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
    assert sel[0]                                   # the oldest request always runs
    assert cta.sum() <= max_ctas
    used = 0
    for i in range(n):
        d = _demand(rows[i], widths[i], cap, work)
        if d <= max_ctas - used:                    # taken in order while its fixed count fits
            assert cta[i] == d
            used += d
        else:
            assert cta[i] == 0

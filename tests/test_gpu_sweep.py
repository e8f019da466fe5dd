"""GPU parity on the Table-3-shaped inputs of the patch-size / search-factor
sweep (Sec. 5.3-5.4): blob, small blob, random shape and long strip, with
9x9 to 17x17 patches and small search factors, bit for bit against the
oracle (a search area with no fully known candidate is NO_SOURCE on both)."""
import numpy as np
import pytest

import oracle
from paper_1403_4238_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_4238_gb300 import api as _api
    return _api


@pytest.mark.parametrize("name,r,alpha", [
    ("walkingman", 4, 0.1), ("walkingman", 8, 0.1), ("river", 6, 0.1), ("divingman", 8, 0.05),
    ("hill", 4, 0.5), ("hill", 8, 1.0), ("hill", 4, 0.1),
])
def test_table3_case_matches_oracle(api, name, r, alpha):
    case = synth.table3_case(name, r)
    ora = oracle.run(case.rgb, case.mask, r, alpha=alpha)
    with api.Inpainter(case.rgb, case.mask, r, alpha=alpha, loop="engine") as ip:
        assert ip.search_rect() == oracle.search_rect(case.mask, r, alpha)
        if ora.status == -4 and ora.iters == 0:
            with pytest.raises(api.InpaintError) as e:
                ip.run()
            assert e.value.code == -4
            return
        rc, n, tr = ip.run(trace=True)
        assert ora.status == 0 and rc == 0 and n == ora.iters
        assert ip.info()["evals"] == ora.evals
        for f in ("px", "py", "qx", "qy", "ssd"):
            assert [t[f] for t in tr] == [int(t[f]) for t in ora.trace], f
        assert np.array_equal(ip.result(), ora.rgb)


def test_sweep_runs_and_tabulates(api):
    from paper_1403_4238_gb300 import sweep

    rows = sweep.sweep(names=["river"], radii=(4, 6), alphas=(0.5, -1.0), log=lambda *a: None)
    assert len(rows) == 4 and all(r["status"] == "ok" for r in rows)
    by = {(r["P"], r["alpha"]): r for r in rows}
    # a smaller search area never does more work
    for P in (9, 13):
        assert 0 < by[(P, 0.5)]["evals"] <= by[(P, -1.0)]["evals"]
    # the exact work of one point equals the oracle's
    case = synth.table3_case("river", 4)
    assert by[(9, 0.5)]["evals"] == oracle.run(case.rgb, case.mask, 4, alpha=0.5).evals
    md = sweep.table(rows)
    assert md.count("| river |") == 2

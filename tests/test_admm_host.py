"""Host-side ADMM controls of the product (the Eq. 10 penalty schedule)
against the oracle's reading of Eq. 10, on random residuals that hit every
branch, and the freeze after the adjustment window."""
import numpy as np

from paper_2405_13943_b300.admm import AdaptivePenalty


def test_adaptive_penalty_matches_oracle_schedule(oracle):
    rng = np.random.default_rng(21)
    rho = [1e4, 1e4, 1e4, 1e3, 1e4]
    ap = AdaptivePenalty(rho, freeze_after=2000)
    want = list(rho)
    branches = set()
    for t in range(0, 3000, 100):
        # squared residuals spread over 8 decades so all three cases occur
        res = 10.0 ** rng.uniform(-6, 2, 10)
        got, factor = ap.update(res, t)
        new = oracle.adaptive_rho(want, res, t)
        for g in range(5):
            branches.add(np.sign(new[g] - want[g]))
        assert got == new, t
        np.testing.assert_allclose(factor, np.array(want) / np.array(new), rtol=1e-15)
        if t >= 2000:
            assert factor == [1.0] * 5
        want = new
    assert branches == {-1.0, 0.0, 1.0}

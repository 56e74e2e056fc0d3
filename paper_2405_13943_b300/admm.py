"""Host side of the ADMM convergence controls (Sec. 3.3).

AdaptivePenalty applies Eq. 10 per property group after a consensus: with
the primal residual r = x - z and the dual residual s = rho (z^t - z^{t-1})
(Eq. 9, both summed over the shared Gaussians by dg_admm_consensus),
rho is multiplied by tau_inc when ||r|| > mu ||s||, divided by tau_dec when
||s|| > mu ||r||, and kept otherwise; adjustment stops after `freeze_after`
iterations (2000 in the paper) so that the fixed-penalty convergence proof
applies from then on.  The paper leaves mu, tau_inc and tau_dec unstated;
the defaults are the usual mu = 10, tau = 2.  Over-relaxation is the alpha
argument of dg_admm_consensus.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple


class AdaptivePenalty:
    def __init__(self, rho: Sequence[float], mu: float = 10.0, tau_inc: float = 2.0, tau_dec: float = 2.0,
                 freeze_after: int = 2000):
        self.rho = [float(r) for r in rho]
        self.mu, self.tau_inc, self.tau_dec, self.freeze_after = mu, tau_inc, tau_dec, freeze_after

    def update(self, residuals: Sequence[float], t: int) -> Tuple[List[float], List[float]]:
        """residuals: the 10 sums of dg_admm_consensus (squared primal per
        group, then squared dual per group).  Returns (new rho, factor to
        apply to the scaled duals u of each group)."""
        old = list(self.rho)
        if t < self.freeze_after:
            for g in range(5):
                r = math.sqrt(max(float(residuals[g]), 0.0))
                s = math.sqrt(max(float(residuals[5 + g]), 0.0))
                if r > self.mu * s:
                    self.rho[g] = old[g] * self.tau_inc
                elif s > self.mu * r:
                    self.rho[g] = old[g] / self.tau_dec
        factor = [o / n for o, n in zip(old, self.rho)]
        return list(self.rho), factor

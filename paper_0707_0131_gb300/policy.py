"""When to stop Incremental eigCG and switch to init-CG (Sec. 5.3).

The paper observes that the largest gains come from the first right-hand sides solved
with Incremental eigCG and that the number worth solving that way grows with the total
number of right-hand sides; it suggests monitoring the improvement at run time.  This
module does that with a cost model in units of CG iterations:

* an eigCG solve costs `eigcg_overhead` times its CG iterations (window upkeep and
  restarts) plus `grow_cost` for adding its Ritz vectors to the basis;
* an init-CG solve costs its CG iterations;
* the iteration count falls with every basis growth, by amounts that shrink roughly
  geometrically (the basis first captures the smallest, most harmful eigenvalues).

After each eigCG solve, with iteration counts n_1 .. n_i observed, the last decrease
d = n_(i-1) - n_i and its ratio rho = d / (n_(i-2) - n_(i-1)) predict the iterations
with the current basis, n = n_i - rho d, and the saving of one more growth, g = rho^2 d.
Solving the next right-hand side with eigCG instead of init-CG pays when the remaining
R - 1 solves after it save more than it costs extra:

    (R - 1) g  >  (eigcg_overhead - 1) n + grow_cost.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass
class SwitchPolicy:
    total_rhs: int
    eigcg_overhead: float = 1.2
    grow_cost: float = 0.0
    min_eigcg: int = 2          # solves before a trend can be estimated
    iters: list = field(default_factory=list)

    def record(self, iterations: int) -> None:
        """Iterations of the eigCG solve just finished."""
        self.iters.append(int(iterations))

    def predicted(self):
        """(iterations with the current basis, saving of one more growth) or None."""
        n = self.iters
        if len(n) < 2:
            return None
        d = n[-2] - n[-1]
        if d <= 0:
            return float(n[-1]), 0.0
        rho = 0.75  # one decrease seen: assume a slow geometric decay
        if len(n) >= 3 and n[-3] - n[-2] > 0:
            rho = min(max(d / (n[-3] - n[-2]), 0.0), 0.95)
        return max(n[-1] - rho * d, 1.0), rho * rho * d

    def use_eigcg(self) -> bool:
        """True: solve the next right-hand side with (Incremental) eigCG."""
        i = len(self.iters)
        remaining = self.total_rhs - i
        if remaining <= 1:
            return False
        if i < self.min_eigcg:
            return True
        it, gain = self.predicted()
        return (remaining - 1) * gain > (self.eigcg_overhead - 1.0) * it + self.grow_cost


def total_cost(iters_by_basis, total_rhs: int, k: int, eigcg_overhead: float, grow_cost: float) -> float:
    """Cost (CG-iteration units) of solving total_rhs right-hand sides with k eigCG solves
    first: iters_by_basis(j) = iterations with the basis grown from j eigCG solves."""
    c = sum(eigcg_overhead * iters_by_basis(j) + grow_cost for j in range(k))
    return c + (total_rhs - k) * iters_by_basis(k)

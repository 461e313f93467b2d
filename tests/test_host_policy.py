"""The eigCG -> init-CG switch policy against the exact optimum of its own cost model.

Synthetic iteration counts n(j) = c + a exp(-j / tau) (iterations after j basis
growths: a fast initial fall that saturates, as in the paper's Fig. 9/10 runs).  For
each total number of right-hand sides the online policy, which only sees the counts of
the solves already made, must reach a total cost within 2% of the minimum over k (the
cost is flat near its minimum, so the chosen k itself may differ by several); the number
of eigCG solves it chooses must not decrease as the total grows (the trend of the
paper's table in Sec. 5.3).
"""
import math

import pytest

from paper_0707_0131_gb300.policy import SwitchPolicy, total_cost


def _run(policy, iters_by_basis):
    k = 0
    while policy.use_eigcg() and k < policy.total_rhs:
        policy.record(iters_by_basis(k))
        k += 1
    return k


@pytest.mark.parametrize("c,a,tau", [(60, 800, 3.0), (120, 600, 5.0), (40, 1200, 2.0)])
@pytest.mark.parametrize("overhead,grow", [(1.2, 0.0), (1.3, 20.0)])
def test_policy_near_optimum(c, a, tau, overhead, grow):
    f = lambda j: c + a * math.exp(-j / tau)  # noqa: E731
    chosen = []
    for total in (6, 12, 24, 32, 48, 96):
        costs = [total_cost(f, total, k, overhead, grow) for k in range(total + 1)]
        k_opt = min(range(total + 1), key=lambda k: costs[k])
        k = _run(SwitchPolicy(total, overhead, grow), f)
        assert costs[k] <= 1.02 * costs[k_opt], (total, k, k_opt, costs[k], costs[k_opt])
        chosen.append(k)
    assert chosen == sorted(chosen), chosen


def test_policy_edge_cases():
    # one right-hand side: nothing to gain from growing a basis
    assert not SwitchPolicy(1).use_eigcg()
    # a flat iteration history stops the eigCG phase as soon as a trend is seen
    p = SwitchPolicy(50)
    for _ in range(2):
        assert p.use_eigcg()
        p.record(300)
    assert not p.use_eigcg()


def test_serving_worker_switch():
    """The serving worker grows the basis while the policy (with an expected request count)
    says so and never returns to eigCG; without a count it fills basis_max."""
    from paper_0707_0131_gb300.serving import OpSpec, _Worker

    f = lambda j: 60 + 800 * math.exp(-j / 3.0)  # noqa: E731
    for expected, cap in [(24, 400), (0, 100)]:
        spec = OpSpec(key="k", dims=(4, 4, 4, 4), m_q=0.1, gauge=None, nev=10, basis_max=cap,
                      expected_requests=expected)
        w = _Worker(None, spec)
        size, solves = 0, 0
        while w.use_eigcg(size):
            if w.policy is not None:
                w.policy.record(f(solves))
            size += spec.nev
            solves += 1
        assert not w.use_eigcg(0)  # the eigCG phase does not come back
        if expected:
            costs = [total_cost(f, expected, k, 1.2, 0.0) for k in range(expected + 1)]
            assert costs[solves] <= 1.02 * min(costs) and size < cap, (solves, size)
        else:
            assert size == cap
        w.q.put(None)

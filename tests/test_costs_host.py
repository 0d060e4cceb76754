"""The per-kernel algorithmic cost table bench.py divides by: every entry
names a kernel the library reports, and the cycle totals stay the figures
the design documents (a change to a kernel's data flow must come with its
cost)."""
import itertools

import pytest

from paper_2209_01983_gb300 import costs


@pytest.fixture(scope="module")
def names():
    from paper_2209_01983_gb300 import sale
    return {sale.sale_kernel_name(i).decode() for i in range(sale.sale_kernel_count())}


def test_every_cost_entry_is_a_library_kernel(names):
    for prec, jit, order, to, hg in itertools.product(("fp64", "fp32_mixed"), (True, False), (1, 2), (1, 2),
                                                      (False, True)):
        t = costs.table(prec, "ale", jitter=jit, order=order, time_order=to, hourglass=hg)
        missing = sorted(k for k in t if k not in names)
        assert not missing, (prec, jit, order, to, hg, missing)
        for k, (unit, b, f) in t.items():
            assert unit in ("cell", "node") and b > 0 and f >= 0, k
    assert not sorted(k for k in costs.table("fp64", "general") if k not in names)
    # several materials: the general kernels, each entry at least its single-material cost
    assert "ale_hourglass" in costs.table("fp64", "ale", hourglass=True, nmat=2)
    for nmat, path in itertools.product((2, 3, 4), ("general", "ale")):
        t, base = costs.table("fp64", path, nmat=nmat), costs.table("fp64", path)
        assert set(t) == set(base) and not sorted(k for k in t if k not in names)
        assert all(t[k][1] >= base[k][1] for k in t) and sum(v[1] for v in t.values()) > sum(v[1] for v in base.values())


def test_cycle_totals():
    assert costs.cycle_cost("fp64") == (1608, 627)
    assert costs.cycle_cost("fp32_mixed", jitter=True) == (588, 957)
    assert costs.cycle_cost("fp32_mixed", jitter=False) == (332, 2521)

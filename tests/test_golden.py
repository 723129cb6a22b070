"""Paper-printed values (tests/golden/, each file cites its table)."""
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_table5_matvec_identity():
    """The matvec counter of the solver reports iters * 2 + 2 * cg_iters
    (one A and one A^T per ADMM iteration, two per CG step); the paper's
    printed totals obey the same identity up to the rounding of the printed
    average CG count (0.05 per iteration, two products per CG step)."""
    rows = read_table("table5_random_socp.txt")
    assert len(rows) == 3
    for _name, iters, avg_cg, mults in rows:
        iters, avg_cg, mults = int(iters), float(avg_cg), int(mults)
        predicted = iters * (2 + 2 * avg_cg)
        assert abs(predicted - mults) <= iters * 2 * 0.05 + 1

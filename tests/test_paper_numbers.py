"""The only numbers the paper prints are Table 1's Gflops (tests/golden): the benchmark's
vs_baseline divides by the paper's best sustained CG figure on this lattice."""
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COLS = ["dw_single", "m5_single", "dw_double", "m5_double", "cg_mixed"]


def table1():
    rows = {}
    for ln in open(os.path.join(ROOT, "tests", "golden", "table1_gflops_16x16x16x32_Ns16.txt")):
        if ln.strip() and not ln.startswith("#"):
            dev, *vals = ln.split()
            rows[dev] = dict(zip(COLS, map(float, vals)))
    return rows


def test_table_is_complete():
    t = table1()
    assert set(t) == {"GTX285", "GTX480", "C1060", "C2050"}
    assert all(len(r) == 5 for r in t.values())


def test_benchmark_divides_by_the_papers_best_cg_figure():
    import bench
    t = table1()
    best = max(r["cg_mixed"] for r in t.values())
    assert best == t["GTX480"]["cg_mixed"] == bench.PAPER_BEST_GFLOPS

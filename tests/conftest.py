import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Parity records of the GPU tests: per test, the largest error against
    the bar (the term-scale measure, 1e-12 for conserved variables and face
    fields, 1e-10 for primitives, P against its recovery scale) and, beside
    it, the plain measure max|a - b| / max(|b|, 1e-10 max|b|) of each field;
    tie faces taken down the GPU's branch and FOFC flags taken over from the
    GPU (each checked to sit within rounding of its decision).  No cell is
    left out of a comparison."""
    try:
        from tests import gpu_util as U
    except Exception:
        return
    if not U.REPORT:
        return
    tr = terminalreporter
    tr.section("parity records (bar measure | plain measure, max over fields and calls)")
    for node, r in sorted(U.REPORT.items()):
        cons = [k for k in r["bar"] if k.startswith(("cons", "bf"))]
        prim = [k for k in r["bar"] if k in ("rho", "w1", "w2", "w3")]
        pl_c = [k for k in r["plain"] if k.startswith(("cons", "bf"))]
        pl_p = [k for k in r["plain"] if k.startswith("prim")]
        def f(d, ks):
            if not ks:
                return "0"
            k = max(ks, key=lambda x: d[x])
            return f"{d[k]:.2e} ({k})"
        tr.write_line(
            f"{node}: calls {r['calls']}; cons+faceB bar {f(r['bar'], cons)} | plain {f(r['plain'], pl_c)}; "
            f"prims bar {f(r['bar'], prim)}, P/scale {r['bar'].get('P/bar', 0.0):.2f} | plain "
            f"{f(r['plain'], pl_p)}; tie faces on the GPU's branch {r['ties']}; FOFC flags taken over "
            f"{r['flips']}; cells excluded 0")

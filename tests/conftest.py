import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libdarb.so")


def pytest_terminal_summary(terminalreporter):
    """Totals of the parity statistics the GPU tests record (nothing when they did not run)."""
    mod = sys.modules.get("gpu_helpers")
    if mod is None:
        return
    tr = terminalreporter
    if mod.GRAD_STATS:
        n = sum(s[1] for s in mod.GRAD_STATS)
        rel = sum(s[2] for s in mod.GRAD_STATS)
        floor = sum(s[3] for s in mod.GRAD_STATS)
        worst = max(mod.GRAD_STATS, key=lambda s: s[3] / max(s[1], 1))
        tr.write_line(f"gradient parity: {n} nonzero reference elements in {len(mod.GRAD_STATS)} comparisons; "
                      f"{rel} ({100.0 * rel / max(n, 1):.3f}%) within 1e-3 relative alone, {floor} "
                      f"({100.0 * floor / max(n, 1):.3f}%) only through the 1e-4 max floor "
                      f"(largest share: {worst[0]}, {worst[3]} of {worst[1]})")
    for st in mod.GEOM64_STATS:
        tr.write_line("fp64 geometry: " + ", ".join(f"{k}={v}" for k, v in st.items()))

"""Host-side checks of bench.py's reporting choices (no GPU)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_headline_mode_is_one_that_meets_the_dissipation_target():
    """The mode bench.py reports as its headline value is one whose GPU test
    asserts the method's dissipation-rate target against the oracle."""
    from test_gpu_modes import MODES, DISS_TARGET
    bench = _bench()
    enc, _, bound_diss, kind = MODES[bench.HEADLINE]
    assert kind == "target" and bound_diss <= DISS_TARGET, bench.HEADLINE
    assert bench.mode_config(__import__("paper_2505_20911_b300"), 256,
                             bench.HEADLINE).encoding == enc

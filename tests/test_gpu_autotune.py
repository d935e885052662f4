"""The option search of the chosen form (leaf size, inner order) on a small
drawing: every candidate is timed, checked against the FP64 reference, and
the fastest accurate one is returned."""
import pytest

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu


def test_autotune_picks_an_accurate_candidate(dcmod, cuda_ok):
    from paper_2311_14312_gb300 import autotune
    d = drawing_by_name("mixed16")
    best, table = autotune.autotune(d, [(0.0, 0.0, 1.0, 1.0, 64, 64), (0.2, 0.3, 0.5, 0.6, 40, 24)],
                                    leaf_sizes=(16, 32), p_inners=(10, 12), repeats=1)
    for opts, ms, err in table:
        print(opts["leaf_size"], opts["p_inner"], ms, f"{err:.2e}")
    assert len(table) == 4
    assert best is not None
    chosen = [t for t in table if t[0] == best][0]
    assert chosen[2] <= 1e-5 and chosen[1] == min(t[1] for t in table if t[1] is not None)

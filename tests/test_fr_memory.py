"""The memory-transfer model of the flux-reconstruction steps against Table
mem_usage (Sec. 4) as printed (tests/golden/fr_mem_usage.txt).

Every T and Gamma matches the printed two decimals, except step 4 at k = 4
and 5, printed as the k = 3 figure (2.50 KiB) where 2 ns np FP32 values give
4.88 and 8.44 KiB.  The printed totals sum the printed step-4 figures; the
weighted Gamma and the predicted gains (20.1, 20.6, 21.0 %) come out of the
model's own step 4, which pins that reading.
"""
import os

import pytest

from paper_2003_02633_gb300 import fr_memory as M

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fr_mem_usage.txt")
KS = (3, 4, 5)


def _printed():
    rows, total, gain = {}, None, None
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "total":
            total = [float(x) for x in f[1:]]
        elif f[0] == "gain":
            gain = [float(f[1]), float(f[3]), float(f[5])]
        else:
            rows[int(f[0])] = [float(x) for x in f[1:]]
    return rows, total, gain


def _close(model, printed):
    # the table rounds to two decimals
    return abs(model - printed) <= 0.005 + 1e-9


@pytest.mark.parametrize("ki", range(3))
def test_steps_match_printed_table(ki):
    k = KS[ki]
    rows, _, _ = _printed()
    model = M.table(k)
    for step, t, g in model:
        pt, pg = rows[step][2 * ki], rows[step][2 * ki + 1]
        if step == 4 and k > 3:
            assert pt == rows[4][0]              # the k = 3 figure, repeated
            ns, _ = M.points(k)
            assert t == pytest.approx(2 * ns * M.NP * 4 / 1024)
            continue
        assert _close(t, pt), (k, step, t, pt)
        assert _close(g, pg), (k, step, g, pg)


@pytest.mark.parametrize("ki", range(3))
def test_totals_and_predicted_gain(ki):
    k = KS[ki]
    _, total, gain = _printed()
    t_printed, _ = M.totals(k, printed_step4=True)
    assert _close(t_printed, total[2 * ki])
    _, g = M.totals(k)
    assert _close(g, total[2 * ki + 1])
    assert abs(100 * (1 - g) - gain[ki]) <= 0.05 + 1e-9
    # the printed step 4 would give other gains at k = 4, 5
    if k > 3:
        _, g_printed = M.totals(k, printed_step4=True)
        assert abs(100 * (1 - g_printed) - gain[ki]) > 0.05


def test_compressible_steps_are_the_highlighted_ones():
    # Table fr_nse highlights n_f (step 2), the gradient tensors (5-9), the
    # metric terms (8, 9) and the flux (9-11)
    assert M.compressible_steps(3) == [2, 5, 6, 7, 8, 9, 10, 11]


def test_row_bytes():
    # a compressed row is 8 bytes against 12 in FP32 (Sec. 2): Gamma 2/3 for a
    # step that moves only rows (step 7)
    for k in KS:
        assert M.step_bytes(k, 7, True) * 3 == M.step_bytes(k, 7) * 2

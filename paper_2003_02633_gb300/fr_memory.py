"""Memory-transfer model of the flux-reconstruction right-hand side (Sec. 4,
Table fr_nse and Table mem_usage): the bytes each of the twelve steps reads and
writes per hexahedral element, with every array in FP32, and the same with the
compressible 3-vector rows (the blue terms of Table fr_nse) stored as 64-bit
words instead of three FP32 components.

Per element of degree k: ns = (k + 1)^3 solution points, nf = 6 (k + 1)^2 flux
points, np = 5 equations.  A scalar field at the solution points is ns * np
FP32 values; a gradient or flux tensor is ns * np rows of three components,
compressed row by row (Eq. eulerF); a metric J is three rows per point; a
normal one row per flux point.

Readings where the table does not follow from Table fr_nse's inputs and
outputs alone (the model reproduces the printed figures with them):
  * step 8 moves one more nf * np FP32 array than its listed operands: read as
    the read-modify-write of the interface flux, the common inviscid flux of
    step 2 being read and n.(F_inv - F_vis) written (the input of step 11);
  * step 12 moves three ns * np arrays (the correction, the divergence and the
    result at the solution points);
  * step 4 is printed as 2.50 KiB for k = 4 and 5, the k = 3 value; the model
    gives 4.88 and 8.44 KiB (2 ns np FP32 values, like the other k), and
    `table()` can return either.  The printed total T sums the printed
    figures, while the printed weighted Gamma and the predicted gains (20.1,
    20.6, 21.0 %) come out only with the model's figures: a typo in the step-4
    cells.
"""
from __future__ import annotations

from dataclasses import dataclass

FP32 = 4          # bytes of one FP32 value
WORD = 8          # bytes of one compressed 3-vector row
NP = 5            # equations (Navier-Stokes: rho, rho u, rho v, rho w, E)


@dataclass(frozen=True)
class Operand:
    """One array a step reads or writes: `per` rows per element, each either a
    scalar (comps = 1) or a 3-vector row (comps = 3); `comp` marks the rows
    Table fr_nse highlights as compressible."""
    name: str
    per: int
    comps: int
    comp: bool = False

    def bytes(self, compressed: bool) -> int:
        if compressed and self.comp:
            assert self.comps == 3
            return self.per * WORD
        return self.per * self.comps * FP32


def points(k: int) -> tuple[int, int]:
    """(ns, nf) of a degree-k hexahedron with tensor-product points."""
    q = k + 1
    return q ** 3, 6 * q * q


def steps(k: int) -> dict[int, list[Operand]]:
    """The operands of each step of Table fr_nse for degree k."""
    ns, nf = points(k)
    n = NP
    return {
        1: [Operand("q^s", ns * n, 1), Operand("q^f", nf * n, 1)],
        2: [Operand("q^f", nf * n, 1), Operand("n_f", nf, 3, True),
            Operand("n.F^I_inv", nf * n, 1)],
        3: [Operand("q^f", nf * n, 1), Operand("w^I", nf * n, 1)],
        4: [Operand("q^s", ns * n, 1), Operand("w^s", ns * n, 1)],
        5: [Operand("w^s", ns * n, 1), Operand("grad w^s", ns * n, 3, True)],
        6: [Operand("grad w^s", ns * n, 3, True), Operand("w^I", nf * n, 1),
            Operand("grad w^c", ns * n, 3, True)],
        7: [Operand("grad w^c", ns * n, 3, True), Operand("grad w^f", nf * n, 3, True)],
        8: [Operand("grad w^f", nf * n, 3, True), Operand("n_f", nf, 3, True),
            Operand("J_f", nf * 3, 3, True), Operand("|J_f|", nf, 1),
            Operand("q^f", nf * n, 1), Operand("n.F^I_inv (read)", nf * n, 1),
            Operand("n.(F^I_inv - F^I_vis)", nf * n, 1)],
        9: [Operand("grad w^s", ns * n, 3, True), Operand("J_s", ns * 3, 3, True),
            Operand("|J_s|", ns, 1), Operand("q^s", ns * n, 1),
            Operand("F^s", ns * n, 3, True)],
        10: [Operand("F^s", ns * n, 3, True), Operand("div F^s", ns * n, 1)],
        11: [Operand("F^s", ns * n, 3, True), Operand("n.(F^I_inv - F^I_vis)", nf * n, 1),
             Operand("F^fc", nf * n, 1)],
        12: [Operand("F^fc", ns * n, 1), Operand("div F^s", ns * n, 1),
             Operand("div F^c", ns * n, 1)],
    }


# Step 4 as printed for k = 4 and 5 (the k = 3 figure), in bytes.
PRINTED_STEP4_BYTES = 2560


def step_bytes(k: int, step: int, compressed: bool = False) -> int:
    """Bytes moved per element by one step."""
    return sum(op.bytes(compressed) for op in steps(k)[step])


def table(k: int, printed_step4: bool = False) -> list[tuple[int, float, float]]:
    """Rows (step, T in KiB, Gamma) of Table mem_usage for degree k.  With
    `printed_step4`, step 4 takes the paper's printed 2.50 KiB."""
    rows = []
    for s in range(1, 13):
        t = step_bytes(k, s)
        c = step_bytes(k, s, compressed=True)
        if s == 4 and printed_step4:
            t = c = PRINTED_STEP4_BYTES
        rows.append((s, t / 1024.0, c / t))
    return rows


def totals(k: int, printed_step4: bool = False) -> tuple[float, float]:
    """(total T in KiB, byte-weighted Gamma) over the twelve steps: the last row
    of Table mem_usage.  1 - Gamma is the predicted gain of Sec. 4 for a
    memory-bound right-hand side."""
    rows = table(k, printed_step4)
    t = sum(r[1] for r in rows)
    c = sum(r[1] * r[2] for r in rows)
    return t, c / t


def compressible_steps(k: int) -> list[int]:
    """The steps with at least one compressible operand."""
    return [s for s, ops in steps(k).items() if any(op.comp for op in ops)]

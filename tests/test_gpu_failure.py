"""Failure paths of the GPU code, made to happen without a GPU fault:

* every wait between the decoding and the accumulating warps of the CUDA-core
  flux-divergence kernel is bounded; with the bound set to one cycle an
  ordinary wait runs out, the blocks leave (copies completed), and
  ivc_flux_divergence_check reports IVC_ERR_TIMEOUT; with the bound restored
  the next launch is correct and reports IVC_OK (the context stays usable);
* the batched kernels check every work-list entry before touching memory: a
  plan whose workspace work list is overwritten (every field's first tile
  set to 0, so most tiles name ranges past their field's end) reads and writes
  nothing out of range and reports IVC_ERR_ARG through ivc_plan_status; a
  fresh plan afterwards gives the oracle's words."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2003_02633_gb300 import ivc, synth  # noqa: E402
from parity_util import formats  # noqa: E402

DEV = "cuda:0"


def _fdiv_inputs(ne=2000, order=3, nvars=5):
    fo, fg = formats("primary")
    F = synth.tgv_euler_flux(elements_per_axis=16, order=order, elements=ne).numpy()[:, :nvars]
    F = np.ascontiguousarray(F)
    ns = F.shape[0]
    w = O.compress(fo, F.reshape(-1, 3)).reshape(ns, nvars, ne)
    Wd = torch.from_numpy(w.view(np.int64)).to(DEV)
    D = torch.from_numpy(synth.fr_hex_operator(order, 2 * math.pi / 16)).to(DEV)
    return fg, Wd, D


def test_fdiv_wait_runs_out_and_recovers():
    fg, Wd, D = _fdiv_inputs()
    L = ivc.load()
    L.ivc_set_flux_divergence_wait_limit(0)
    ref = ivc.flux_divergence(fg, Wd, D, simt=True)     # default bound: completes
    assert L.ivc_flux_divergence_check() == ivc.IVC_OK
    out = torch.zeros_like(ref)
    try:
        assert L.ivc_set_flux_divergence_wait_limit(1) == ivc.IVC_OK
        ivc.flux_divergence(fg, Wd, D, out=out, simt=True)
        torch.cuda.synchronize()
        assert L.ivc_flux_divergence_check() == ivc.IVC_ERR_TIMEOUT
        assert L.ivc_flux_divergence_check() == ivc.IVC_OK      # reported once
    finally:
        L.ivc_set_flux_divergence_wait_limit(0)
    # bound restored: the same launch completes and gives the same result
    # (the kernel's order of operations is fixed)
    ivc.flux_divergence(fg, Wd, D, out=out, simt=True)
    assert L.ivc_flux_divergence_check() == ivc.IVC_OK
    assert torch.equal(out, ref)


def _fields(fo, fg, lens, seed):
    out = []
    for i, m in enumerate(lens):
        a, b = synth.roundtrip_inputs(m, seed=seed + i)
        a, b = a[:m], b[:m]
        wa, wb = O.compress(fo, a), O.compress(fo, b)
        out.append((torch.from_numpy(wa.view(np.int64)).to(DEV),
                    torch.from_numpy(wb.view(np.int64)).to(DEV),
                    torch.full((m,), -1, dtype=torch.int64, device=DEV), 0.0, wa, wb))
    return out


@pytest.mark.parametrize("name", ["primary", "tanh"])
def test_batched_corrupted_work_list_is_reported(name):
    fo, fg = formats(name)
    lens = [5000, 70, 12000, 1, 4096, 9000]
    fl = _fields(fo, fg, lens, seed=300)
    fields = [f[:4] for f in fl]
    cfg = ivc.ivc_launch_config(128, 2, 1024, 1)
    plan = ivc.BatchedPlan(fg, ivc.IVC_OP_ADD, fields, cfg=cfg)
    # workspace layout: field table (40 B per field, padded to 256 B), then the
    # per-field first-tile prefix (nfields + 1 int64)
    base = (plan.workspace.data_ptr() + 255) // 256 * 256 - plan.workspace.data_ptr()
    off = base + (40 * len(lens) + 255) // 256 * 256
    plan.workspace[off:off + 8 * (len(lens) + 1)].zero_()
    plan.launch(graph=False)
    assert plan.status() == ivc.IVC_ERR_ARG
    plan.close()
    torch.cuda.synchronize()
    # a fresh plan on the same fields is correct (the context is usable)
    plan = ivc.BatchedPlan(fg, ivc.IVC_OP_ADD, fields, cfg=cfg)
    plan.launch()
    assert plan.status() == ivc.IVC_OK
    plan.close()
    for (da, db, dc, _, wa, wb) in fl:
        got = dc.cpu().numpy().view(np.uint64)
        want = O.add(fo, wa, wb)
        assert int(np.sum(got != want)) <= 1

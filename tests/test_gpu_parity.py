"""GPU parity: the CUDA path (through the C ABI) against the oracle.

Sizes span many blocks and a ragged tail; inputs are seeded (``synth``); the
oracle's inputs and expected values never come from the CUDA path: where a
fused operation needs compressed inputs, the oracle compresses the same FP32
vectors itself and the GPU is given the oracle's words.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2003_02633_gb300 import ivc, synth  # noqa: E402
from parity_util import (FORMATS, allowed_mismatches, check_decoded, check_words,  # noqa: E402
                         formats)

DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _words_dev(w):
    return _dev(np.asarray(w, np.uint64).view(np.int64))


def _host_words(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def c0():
    """Round trip + add workload: 2^20 vectors per operand plus 64 edge vectors."""
    a, b = synth.roundtrip_inputs(1 << 20, seed=0)
    return a, b


def test_compress_config0(c0):
    fo, fg = formats("primary")
    for x in c0:
        wg = _host_words(ivc.compress(fg, _dev(x)))
        check_words(fo, x, wg, O.compress(fo, x), "compress")


def test_decompress_config0(c0):
    fo, fg = formats("primary")
    w = O.compress(fo, c0[0])
    got = ivc.decompress(fg, _words_dev(w)).cpu().numpy()
    exact = check_decoded(got, O.decompress(fo, w), "decompress")
    assert exact > 0.9999


def test_decompress_random_words():
    fo, fg = formats("primary")
    w = synth.random_words(1 << 18, seed=3)
    got = ivc.decompress(fg, _words_dev(w)).cpu().numpy()
    exact = check_decoded(got, O.decompress(fo, w), "decompress random words")
    assert exact > 0.9999


def test_add_config0(c0):
    fo, fg = formats("primary")
    a, b = c0
    wa, wb = O.compress(fo, a), O.compress(fo, b)
    want = O.add(fo, wa, wb)
    with np.errstate(invalid="ignore", over="ignore"):
        pre = O.decompress(fo, wa) + O.decompress(fo, wb)
    got = _host_words(ivc.add(fg, _words_dev(wa), _words_dev(wb)))
    check_words(fo, pre, got, want, "add")


def test_add_in_place_and_misaligned(c0):
    fo, fg = formats("primary")
    a, b = c0[0][:100001], c0[1][:100001]
    wa, wb = O.compress(fo, a), O.compress(fo, b)
    want = O.add(fo, wa, wb)
    with np.errstate(invalid="ignore", over="ignore"):
        pre = O.decompress(fo, wa) + O.decompress(fo, wb)
    da, db = _words_dev(wa), _words_dev(wb)
    ivc.add(fg, da, db, out=da)                    # in place, odd n (ragged tail)
    check_words(fo, pre, _host_words(da), want, "add in place")
    # offset by one word: 8-byte but not 16-byte aligned -> scalar path
    buf = torch.zeros(3 * (len(wa) + 1), dtype=torch.int64, device=DEV)
    x, y, z = buf[1:1 + len(wa)], buf[len(wa) + 2:2 * len(wa) + 2], buf[2 * len(wa) + 2:]
    x.copy_(_words_dev(wa))
    y.copy_(_words_dev(wb))
    ivc.add(fg, x, y, out=z[:len(wa)])
    check_words(fo, pre, _host_words(z[:len(wa)]), want, "add misaligned")


def test_axpy_config0(c0):
    fo, fg = formats("primary")
    a, b = c0
    wx, wy = O.compress(fo, a), O.compress(fo, b)
    alpha = np.float32(0.7)
    want = O.axpy(fo, alpha, wx, wy)
    dx, dy = O.decompress(fo, wx).astype(np.float64), O.decompress(fo, wy).astype(np.float64)
    with np.errstate(invalid="ignore", over="ignore"):
        pre = (np.float64(alpha) * dx + dy).astype(np.float32)  # one rounding of the exact fma
    y = _words_dev(wy)
    ivc.axpy(fg, alpha, _words_dev(wx), y)
    check_words(fo, pre, _host_words(y), want, "axpy")


def test_pointwise_update_tgv():
    fo, fg = formats("primary")
    v, f, rho = synth.tgv_fields(elements_per_axis=12)   # 12^3 elements x 64 points
    wv, wf = O.compress(fo, v), O.compress(fo, f)
    dt = np.float32(1e-3)
    vo, mo = O.update(fo, dt, wv, wf, rho, want_m=True)
    vg, mg = ivc.pointwise_update(fg, dt, _words_dev(wv), _words_dev(wf), rho=_dev(rho),
                                  m_out=torch.empty(len(wv), dtype=torch.int64, device=DEV))
    dv = O.decompress(fo, wv).astype(np.float64)
    df = O.decompress(fo, wf).astype(np.float64)
    pre = (np.float64(dt) * df + dv).astype(np.float32)
    check_words(fo, pre, _host_words(vg), vo, "update v")
    check_words(fo, rho[:, None] * pre, _host_words(mg), mo, "update m")


def test_pointwise_update_momentum_any_rho():
    """m = encode(rho * v_new): the fast kernel takes m's angle estimates from
    v_new's (m points where v_new does when rho > 0), with a wider ambiguity
    band, and sends m to the generic encoder when rho is not positive and
    finite or v_new lies outside the fast window.  Random directions and
    magnitudes, edge vectors, and densities from 10^U(-3, 3) mixed with 0,
    -0, negative, tiny, huge, Inf and NaN values, against the oracle."""
    fo, fg = formats("primary")
    v, f = synth.roundtrip_inputs((1 << 18) + 5, seed=61)
    rng = np.random.default_rng(62)
    rho = (10.0 ** rng.uniform(-3, 3, v.shape[0])).astype(np.float32)
    special = np.float32([0.0, -0.0, -1.0, -2.5e3, 1e-38, 3e38, np.inf, -np.inf, np.nan, 1e-45])
    idx = rng.choice(v.shape[0], 4000, replace=False)
    rho[idx] = special[rng.integers(0, len(special), len(idx))]
    with np.errstate(invalid="ignore", over="ignore"):
        wv, wf = O.compress(fo, v), O.compress(fo, f)
        dt = np.float32(1e-3)
        vo, mo = O.update(fo, dt, wv, wf, rho, want_m=True)
        dv = O.decompress(fo, wv).astype(np.float64)
        df = O.decompress(fo, wf).astype(np.float64)
        pre = (np.float64(dt) * df + dv).astype(np.float32)
        pre_m = (rho[:, None].astype(np.float64) * pre).astype(np.float32)
    vg, mg = ivc.pointwise_update(fg, dt, _words_dev(wv), _words_dev(wf), rho=_dev(rho),
                                  m_out=torch.empty(len(wv), dtype=torch.int64, device=DEV))
    check_words(fo, pre, _host_words(vg), vo, "update v")
    check_words(fo, pre_m, _host_words(mg), mo, "update m, any rho")


def test_soa_layout(c0):
    fo, fg = formats("primary")
    x = c0[0][:70001]
    n, ld = x.shape[0], x.shape[0] + 13
    rows = np.zeros((3, ld), np.float32)
    rows[:, :n] = x.T
    w = torch.empty(n, dtype=torch.int64, device=DEV)
    ivc.compress_soa(fg, _dev(rows), ld, n, w)
    check_words(fo, x, _host_words(w), O.compress(fo, x), "compress soa")
    out = torch.zeros((3, ld), dtype=torch.float32, device=DEV)
    L = ivc.load()
    import ctypes
    st = L.ivc_decompress(ctypes.byref(fg), w.data_ptr(), n, out.data_ptr(), ivc.IVC_SOA, ld,
                          torch.cuda.current_stream().cuda_stream)
    assert st == ivc.IVC_OK
    got = out.cpu().numpy()[:, :n].T
    check_decoded(got, O.decompress(fo, O.compress(fo, x)), "decompress soa")


@pytest.mark.parametrize("name", [k for k in FORMATS if k != "primary"])
def test_formats(name):
    fo, fg = formats(name)
    a, b = synth.roundtrip_inputs(1 << 16, seed=7)
    if name == "tiny":
        a = a / np.float32(16.0)
        b = b / np.float32(16.0)
    wa = _host_words(ivc.compress(fg, _dev(a)))
    check_words(fo, a, wa, O.compress(fo, a), f"{name} compress")
    wa, wb = O.compress(fo, a), O.compress(fo, b)
    check_decoded(ivc.decompress(fg, _words_dev(wa)).cpu().numpy(), O.decompress(fo, wa),
                  f"{name} decompress")
    with np.errstate(invalid="ignore", over="ignore"):
        pre = O.decompress(fo, wa) + O.decompress(fo, wb)
    got = _host_words(ivc.add(fg, _words_dev(wa), _words_dev(wb)))
    check_words(fo, pre, got, O.add(fo, wa, wb), f"{name} add")


def test_tanh_add_axpy_many_iterations():
    """The tanh map's fused add and axpy copy every decoded word's two table
    entries into shared memory one iteration ahead (cp.async, two buffers):
    2^21 + 3 vectors give each warp about a dozen iterations (both buffers
    reused several times, odd tail), against the oracle; axpy in place."""
    fo, fg = formats("tanh")
    a, b = synth.roundtrip_inputs((1 << 21) + 3, seed=71)
    wa, wb = O.compress(fo, a), O.compress(fo, b)
    with np.errstate(invalid="ignore", over="ignore"):
        da, db = O.decompress(fo, wa), O.decompress(fo, wb)
        pre = da + db
        alpha = np.float32(0.7)
        pre_axpy = (np.float64(alpha) * da.astype(np.float64) + db).astype(np.float32)
    got = _host_words(ivc.add(fg, _words_dev(wa), _words_dev(wb)))
    check_words(fo, pre, got, O.add(fo, wa, wb), "tanh add, many iterations")
    y = _words_dev(wb)
    ivc.axpy(fg, alpha, _words_dev(wa), y)
    check_words(fo, pre_axpy, _host_words(y), O.axpy(fo, alpha, wa, wb),
                "tanh axpy in place, many iterations")


@pytest.mark.parametrize("name", ["primary", "L1717", "L1617", "fracsplit"])
def test_decompress_many_iterations(name):
    """The fast decompress copies each word's phi^ table entry into shared
    memory one iteration ahead (cp.async, two buffers): 2^21 + 3 words give
    every thread about a dozen iterations and an odd tail; the decoded
    vectors match the oracle's (within one ulp, bit for bit almost always, as
    for the other decompress tests)."""
    fo, fg = formats(name)
    a, _ = synth.roundtrip_inputs((1 << 21) + 3, seed=73)
    w = O.compress(fo, a)
    with np.errstate(invalid="ignore", over="ignore"):
        want = O.decompress(fo, w)
    got = ivc.decompress(fg, _words_dev(w)).cpu().numpy()
    same = check_decoded(got, want, f"{name} decompress, many iterations")
    assert same > 0.9999, f"{name}: {1 - same:.2e} of the decodes differ from the oracle"


def test_counts_match_oracle():
    fo, fg = formats("primary")
    x = synth.precision_vectors(1 << 16, seed=11)
    x = np.concatenate([x, synth.edge_vectors()])
    counts = torch.zeros(3, dtype=torch.int64, device=DEV)
    w = ivc.compress(fg, _dev(x), counts=counts)
    wo, co = O.compress(fo, x, return_counts=True)
    check_words(fo, x, _host_words(w), wo, "precision compress")
    c = counts.cpu().numpy()
    assert (c[0], c[1], c[2]) == (co["n_overflow"], co["n_underflow"], co["n_nonfinite"])


def test_zero_and_tiny_sizes():
    fo, fg = formats("primary")
    L = ivc.load()
    import ctypes
    s = torch.cuda.current_stream().cuda_stream
    assert L.ivc_add(ctypes.byref(fg), 0, 0, 0, 0, s) == ivc.IVC_OK
    for n in (1, 2, 3, 31, 33, 255, 257, 1023):
        a, b = synth.roundtrip_inputs(n, seed=n)
        a, b = a[:n], b[:n]
        wa, wb = O.compress(fo, a), O.compress(fo, b)
        got = _host_words(ivc.add(fg, _words_dev(wa), _words_dev(wb)))
        with np.errstate(invalid="ignore", over="ignore"):
            pre = O.decompress(fo, wa) + O.decompress(fo, wb)
        check_words(fo, pre, got, O.add(fo, wa, wb), f"add n={n}")
        check_words(fo, a, _host_words(ivc.compress(fg, _dev(a))), wa, f"compress n={n}")


def test_error_statuses_on_device():
    fo, fg = formats("primary")
    L = ivc.load()
    import ctypes
    s = torch.cuda.current_stream().cuda_stream
    x = torch.zeros(16, dtype=torch.int64, device=DEV)
    odd = x.data_ptr() + 4
    assert L.ivc_add(ctypes.byref(fg), odd, x.data_ptr(), x.data_ptr(), 4, s) == ivc.IVC_ERR_ALIGN
    assert L.ivc_add(ctypes.byref(fg), 0, x.data_ptr(), x.data_ptr(), 4, s) == ivc.IVC_ERR_ARG
    torch.cuda.synchronize()


def test_batched_plan_matches_oracle():
    fo, fg = formats("primary")
    lens, win = synth.batched_fields(24, seed=5, scale=1.0 / 64)
    rng = np.random.default_rng(9)
    fields, want, pre = [], [], []
    for i, n in enumerate(lens):
        a = synth.random_vectors(int(n), rng=rng, lo=win[i, 0], hi=win[i, 1])
        b = synth.random_vectors(int(n), rng=rng, lo=win[i, 0], hi=win[i, 1])
        wa, wb = O.compress(fo, a), O.compress(fo, b)
        want.append(O.add(fo, wa, wb))
        pre.append(O.decompress(fo, wa) + O.decompress(fo, wb))
        fields.append((_words_dev(wa), _words_dev(wb),
                       torch.zeros(int(n), dtype=torch.int64, device=DEV), 0.0))
    cfg = ivc.ivc_launch_config(256, 2, 4096, 0)
    plan = ivc.BatchedPlan(fg, ivc.IVC_OP_ADD, fields, cfg=cfg)
    for graph in (True, False, True):
        for f in fields:
            f[2].zero_()
        plan.launch(graph=graph)
        assert plan.status() == ivc.IVC_OK
        for i, f in enumerate(fields):
            check_words(fo, pre[i], _host_words(f[2]), want[i], f"batched field {i}")
    plan.close()


def test_batched_axpy_plan():
    fo, fg = formats("primary")
    rng = np.random.default_rng(21)
    fields, want, pre = [], [], []
    for n in (1, 5000, 77777, 3):
        x = synth.random_vectors(n, rng=rng)
        y = synth.random_vectors(n, rng=rng)
        wx, wy = O.compress(fo, x), O.compress(fo, y)
        want.append(O.axpy(fo, np.float32(0.7), wx, wy))
        dx, dy = O.decompress(fo, wx).astype(np.float64), O.decompress(fo, wy).astype(np.float64)
        pre.append((np.float64(np.float32(0.7)) * dx + dy).astype(np.float32))
        fields.append((_words_dev(wx), None, _words_dev(wy), 0.7))
    plan = ivc.BatchedPlan(fg, ivc.IVC_OP_AXPY, fields)
    plan.launch()
    assert plan.status() == ivc.IVC_OK
    for i, f in enumerate(fields):
        check_words(fo, pre[i], _host_words(f[2]), want[i], f"batched axpy {i}")
    plan.close()


def test_f32_and_half_baselines():
    a, b = synth.roundtrip_inputs(100003, seed=2)
    a, b = a[:100003], b[:100003]
    with np.errstate(invalid="ignore", over="ignore"):
        want = a + b
    got = ivc.f32_add(_dev(a), _dev(b)).cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(got[~np.isnan(want)], want[~np.isnan(want)])
    y = _dev(b)
    ivc.f32_axpy(0.7, _dev(a), y)
    ya = y.cpu().numpy()
    ex = (np.float64(np.float32(0.7)) * a.astype(np.float64) + b.astype(np.float64)).astype(np.float32)
    fin = np.isfinite(ex)
    assert np.array_equal(ya[fin], ex[fin])
    # SoA rows with a leading dimension
    n, ld = 5001, 5008
    rows_a = np.zeros((3, ld), np.float32)
    rows_b = np.zeros((3, ld), np.float32)
    rows_a[:, :n], rows_b[:, :n] = a[:n].T, b[:n].T
    out = torch.zeros((3, ld), dtype=torch.float32, device=DEV)
    ivc.f32_add(_dev(rows_a), _dev(rows_b), out=out, layout=ivc.IVC_SOA, ld=ld, n=n)
    with np.errstate(invalid="ignore", over="ignore"):
        w2 = (rows_a + rows_b)[:, :n]
    g2 = out.cpu().numpy()[:, :n]
    m = np.isfinite(w2)
    assert np.array_equal(g2[m], w2[m])
    small = synth.random_vectors(40001, seed=3, lo=-2, hi=2)
    small_b = synth.random_vectors(40001, seed=4, lo=-2, hi=2)
    for kind, tdt in ((ivc.IVC_F16, torch.float16), (ivc.IVC_BF16, torch.bfloat16)):
        ha = ivc.half_from_f32(kind, _dev(small))
        hb = ivc.half_from_f32(kind, _dev(small_b))
        ta = torch.from_numpy(small).to(tdt)
        tb = torch.from_numpy(small_b).to(tdt)
        assert torch.equal(ha.cpu().view(tdt), ta)
        hc = ivc.half_add(kind, ha, hb)
        want = (ta.float() + tb.float()).to(tdt)
        assert torch.equal(hc.cpu().view(tdt), want)
        back = ivc.half_to_f32(kind, hc).cpu()
        assert torch.equal(back, want.float())


def test_error_stats_match_oracle():
    fo, fg = formats("primary")
    x = synth.random_vectors(200001, seed=12)
    w = O.compress(fo, x)
    xh = O.decompress(fo, w)
    acc = ivc.error_stats(_dev(x), _dev(xh))
    st = ivc.stats_dict(acc.cpu())
    so = O.error_stats(x, xh)
    assert st["n"] == so["n"]
    for k in ("mean", "sd", "max", "mean_rel", "max_rel", "max_ang", "rms_ang", "max_mag_rel",
              "rms_mag_rel"):
        assert np.isclose(st[k], so[k], rtol=1e-9, atol=1e-300), k


def test_tune_returns_a_valid_shape():
    fo, fg = formats("primary")
    a, b = synth.roundtrip_inputs(1 << 18, seed=1)
    wa, wb = _words_dev(O.compress(fo, a)), _words_dev(O.compress(fo, b))
    c = torch.empty_like(wa)
    best = ivc.tune(fg, ivc.IVC_OP_ADD, wa, wb, c)
    assert best.block in (64, 128, 256) and best.blocks_per_sm >= 1
    out = ivc.add(fg, wa, wb, cfg=best)
    want = O.add(fo, O.compress(fo, a), O.compress(fo, b))
    with np.errstate(invalid="ignore", over="ignore"):
        pre = O.decompress(fo, O.compress(fo, a)) + O.decompress(fo, O.compress(fo, b))
    check_words(fo, pre, _host_words(out), want, "add tuned")


def _add_pre(fo, wa, wb):
    """The oracle's pre-quantisation vectors of an add: decoded a + decoded b."""
    with np.errstate(invalid="ignore", over="ignore"):
        return O.decompress(fo, wa) + O.decompress(fo, wb)


@pytest.mark.parametrize("ws_vectors", [1000, 1 << 16])
def test_add_host_streams_chunks(c0, ws_vectors):
    """ivc_add_host: host words through a device workspace of a few chunks
    (ragged last chunk, more chunks than slots) give the oracle's words."""
    fo, fg = formats("primary")
    wa, wb = O.compress(fo, c0[0]), O.compress(fo, c0[1])
    n = wa.shape[0]
    ha = torch.from_numpy(wa.view(np.int64)).pin_memory()
    hb = torch.from_numpy(wb.view(np.int64)).pin_memory()
    hc = torch.zeros(n, dtype=torch.int64).pin_memory()
    ws = torch.empty(3 * 3 * ws_vectors, dtype=torch.int64, device=DEV)
    ivc.add_host(fg, ha, hb, hc, ws)
    torch.cuda.synchronize()
    got = hc.numpy().view(np.uint64)
    exp = O.add(fo, wa, wb)
    dev = _host_words(ivc.add(fg, _words_dev(wa), _words_dev(wb)))
    assert np.array_equal(got, dev)
    check_words(fo, _add_pre(fo, wa, wb), got, exp, "add_host chunks")


def test_add_host_pageable_staged(c0):
    """Pageable host words take the staged path (chunks through the workspace)."""
    fo, fg = formats("primary")
    wa, wb = O.compress(fo, c0[0]), O.compress(fo, c0[1])
    n = wa.shape[0]
    hc = torch.zeros(n, dtype=torch.int64)
    ws = torch.empty(3 * 3 * 4096, dtype=torch.int64, device=DEV)
    ivc.add_host(fg, torch.from_numpy(wa.view(np.int64)), torch.from_numpy(wb.view(np.int64)),
                 hc, ws)
    torch.cuda.synchronize()
    check_words(fo, _add_pre(fo, wa, wb), hc.numpy().view(np.uint64), O.add(fo, wa, wb),
                "add_host pageable")


def test_add_host_pinned_without_workspace(c0):
    fo, fg = formats("primary")
    wa, wb = O.compress(fo, c0[0]), O.compress(fo, c0[1])
    n = wa.shape[0]
    ha = torch.from_numpy(wa.view(np.int64)).pin_memory()
    hb = torch.from_numpy(wb.view(np.int64)).pin_memory()
    hc = torch.zeros(n, dtype=torch.int64).pin_memory()
    ivc.add_host(fg, ha, hb, hc)     # zero-copy: no workspace needed
    torch.cuda.synchronize()
    check_words(fo, _add_pre(fo, wa, wb), hc.numpy().view(np.uint64), O.add(fo, wa, wb),
                "add_host pinned")


def test_add_host_tiny_chunks():
    fo, fg = formats("primary")
    a, b = synth.roundtrip_inputs(101, seed=5)
    wa, wb = O.compress(fo, a), O.compress(fo, b)
    n = wa.shape[0]
    ha = torch.from_numpy(wa.view(np.int64))           # pageable memory also works
    hb = torch.from_numpy(wb.view(np.int64))
    hc = torch.zeros(n, dtype=torch.int64)
    ws = torch.empty(3 * 3 * 2, dtype=torch.int64, device=DEV)   # chunks of 2 vectors
    ivc.add_host(fg, ha, hb, hc, ws)
    torch.cuda.synchronize()
    got = hc.numpy().view(np.uint64)
    check_words(fo, _add_pre(fo, wa, wb), got, O.add(fo, wa, wb), "add_host tiny chunks")

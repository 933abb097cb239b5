"""Moving parents, unweighting and gather (section 4.2: Generate(Mother, ...), "weighted and
unweighted samples") against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1711_05683_b300 as hp  # noqa: E402
import workloads  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = {"f64": 1e-12, "f32": 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_05683_b300 import build as hp_build
    hp_build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [2, 3, 7, 10])
def test_boosted_one_mother(n, dtype):
    rng = np.random.default_rng(40 + n)
    M, masses = workloads.random_decay(rng, n)
    mother = (0.4 * M, -2.5 * M, 1.1 * M)
    nev = 2001
    p, w = hp.generate_boosted(M, masses, nev, 9, mother=mother, dtype=dtype, event_offset=5)
    ref_p, ref_w = oracle.generate_boosted(M, masses, nev, 9, mother=mother, event_offset=5)
    gp = p[:, :, :nev].double().cpu().numpy()
    scale = np.maximum(ref_p[:, 0, :].max(axis=0), M)
    assert (np.abs(gp - ref_p) / scale).max() <= TOL[dtype]
    np.testing.assert_allclose(w.double().cpu().numpy(), ref_w, rtol=TOL[dtype])


@pytest.mark.parametrize("dtype,n", [("f32", 3), ("f32", 6), ("f32", 9), ("f64", 4)])
def test_boosted_generation_independent_of_launch_shape(dtype, n):
    """The moving-parent generator follows the generator's tuned shape (FP32 groups of up to
    four events); every shape gives the same bits, ragged tails included, for one momentum and
    for per-event momenta."""
    rng = np.random.default_rng(70 + n)
    M, masses = workloads.random_decay(rng, n)
    nev = 10_003
    tdt = torch.float32 if dtype == "f32" else torch.float64
    moms = torch.as_tensor(rng.normal(0.0, 3.0 * M, size=(3, nev)), dtype=tdt, device="cuda").contiguous()
    saved = hp.get_launch_config(hp.KERNEL_GENERATE, n, dtype)
    runs = []
    try:
        for block, ept in ((256, 1), (128, 2), (256, 4), (512, 4)):
            hp.set_launch_config(hp.KERNEL_GENERATE, n, dtype, block, ept)
            a = hp.generate_boosted(M, masses, nev, 11, mother=(0.3 * M, 0.0, -1.7 * M), dtype=dtype)
            b = hp.generate_boosted(M, masses, nev, 11, mothers=moms, dtype=dtype, event_offset=3)
            torch.cuda.synchronize()
            runs.append((a, b))
    finally:
        hp.set_launch_config(hp.KERNEL_GENERATE, n, dtype, *saved)
    for (a, b) in runs[1:]:
        for x, y in zip(a + b, runs[0][0] + runs[0][1]):
            assert torch.equal(x[..., :nev], y[..., :nev])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_boosted_per_event_mothers(dtype):
    M, masses = 3.0, (0.2, 0.3, 0.4, 0.5, 0.1)
    nev = 3003
    rng = np.random.default_rng(3)
    moms = rng.normal(0.0, 6.0, size=(3, nev))
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dm = torch.as_tensor(moms, dtype=tdt, device="cuda").contiguous()
    p, _ = hp.generate_boosted(M, masses, nev, 4, mothers=dm, dtype=dtype)
    ref_p, _ = oracle.generate_boosted(M, masses, nev, 4, mothers=dm.double().cpu().numpy())
    scale = np.maximum(ref_p[:, 0, :].max(axis=0), M)
    assert (np.abs(p[:, :, :nev].double().cpu().numpy() - ref_p) / scale).max() <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_unweighting_matches_oracle(dtype):
    """Kept events are those of the oracle's accept-reject, except where u w_max and w differ
    by less than the weights' tolerance (there either decision is correct)."""
    cfg = workloads.B_TO_JPSI_K_PI
    M, masses, n = cfg["M"], cfg["masses"], 3
    nev = 100_003
    p, w = hp.generate(M, masses, nev, 21, dtype=dtype)
    ref_p, ref_w = oracle.generate(M, masses, nev, 21)
    w_max = float(ref_w.max()) * 1.0000001
    idx, used = hp.unweight(n, w, 21, w_max=w_max, dtype=dtype)
    got = np.zeros(nev, dtype=bool)
    got[idx.cpu().numpy()] = True
    acc = oracle.unweight(M, masses, nev, 21, w_max=w_max)
    u = (np.array([oracle.draw(21, e, 3 * n - 4) for e in range(nev)], dtype=np.float64) + 0.5) / 2 ** 32
    band = np.abs(u * w_max - ref_w) <= 4 * TOL[dtype] * ref_w + 1e-300
    assert np.all((got == acc) | band)
    assert np.all(np.diff(idx.cpu().numpy()) > 0)  # strictly increasing, stable order
    # the sample's own maximum as the bound
    idx2, used2 = hp.unweight(n, w, 21, dtype=dtype)
    assert used2 == pytest.approx(float(w.max()), rel=0, abs=0)
    assert 0 < len(idx2) < nev
    # gather: the compacted events are the selected events
    dst, dw = hp.gather(p, w, idx2, dtype=dtype)
    assert torch.equal(dst, p[:, :, idx2]) and torch.equal(dw, w[idx2])


def test_unweighting_is_deterministic_and_chunkable():
    """Accept decisions depend only on (seed, event index, w, w_max): two halves with
    event_offset give the indices of one call."""
    M, masses = 10.0, workloads.sweep_masses(5, True)
    nev = 50_000
    p, w = hp.generate(M, masses, nev, 8, dtype="f64")
    wm = float(w.max())
    a, _ = hp.unweight(5, w, 8, w_max=wm, dtype="f64")
    h = 20_000
    b1, _ = hp.unweight(5, w[:h].contiguous(), 8, w_max=wm, dtype="f64")
    b2, _ = hp.unweight(5, w[h:].contiguous(), 8, w_max=wm, dtype="f64", event_offset=h)
    assert torch.equal(a, torch.cat([b1, b2 + h]))


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_unweighting_sample_maximum_any_alignment(dtype):
    """The sample maximum (16-byte vector loads when the weights are aligned, element loads for
    a misaligned view and the remainder) equals torch's max; the kept indices of an offset
    view are those of the full call shifted, with the same bound."""
    M, masses = 10.0, workloads.sweep_masses(4, True)
    p, w = hp.generate(M, masses, 70_001, 5, dtype=dtype)
    for lo, hi in ((0, 70_001), (1, 70_001), (3, 69_998), (0, 7), (1, 2)):
        v = w[lo:hi]
        _, used = hp.unweight(4, v, 5, dtype=dtype, event_offset=lo)
        assert used == float(v.max())
    wm = float(w.max())
    full, _ = hp.unweight(4, w, 5, w_max=wm, dtype=dtype)
    part, _ = hp.unweight(4, w[1:], 5, w_max=wm, dtype=dtype, event_offset=1)
    assert torch.equal(full[full >= 1], part + 1)


@pytest.mark.parametrize("arith", ["double-float", "native"])
def test_evaluate_on_oracle_events_fp64(arith):
    """The evaluation kernel on the oracle's own events (uploaded) reproduces the oracle's
    values and sums; on GPU-generated events it reproduces the generated-event integral; in
    double-float (the FP64 components split by integer operations) and in native FP64."""
    saved = hp.get_fp64_arith()
    hp.set_fp64_arith(hp.FP64_NATIVE if arith == "native" else hp.FP64_DOUBLE_FLOAT)
    try:
        _evaluate_on_oracle_events_fp64()
    finally:
        hp.set_fp64_arith(saved)


def _evaluate_on_oracle_events_fp64():
    d = workloads.D0_DALITZ
    nev = 3 * 2048 * 5 + 77
    p, w = oracle.generate(d["M"], d["masses"], nev, seed=12)
    vals_ref, sums_ref = oracle.evaluate(p, w, me=1, params=d["params"])
    dp = torch.as_tensor(p, device="cuda").contiguous()
    dw = torch.as_tensor(w, device="cuda").contiguous()
    res, vals = hp.evaluate(dp, dw, me=hp.ME_DALITZ_2BW, params=d["params"], dtype="f64", want_values=True)
    np.testing.assert_allclose(vals.cpu().numpy(), vals_ref, rtol=1e-12)
    np.testing.assert_allclose([res["sum_f"], res["sum_f2"], res["sum_w"], res["sum_w2"]], sums_ref, rtol=1e-12)
    gp, gw = hp.generate(d["M"], d["masses"], nev, 12, dtype="f64")
    res2, _ = hp.evaluate(gp, gw, me=hp.ME_DALITZ_2BW, params=d["params"], dtype="f64")
    ref2 = hp.integrate(d["M"], d["masses"], nev, 12, kin_dtype="f64", me=hp.ME_DALITZ_2BW, params=d["params"])
    assert res2["sum_f"] == pytest.approx(ref2["sum_f"], rel=1e-12)
    assert res2["sum_w"] == pytest.approx(ref2["sum_w"], rel=1e-12)


def fp32_dalitz_value_bound(ev, w, params):
    """Per-event bound on |f_FP32 - f| for f = w |A|^2, A = BW(s12; a) + c BW(s23; b), evaluated
    in FP32 from the same stored events (ev [3, 4, n] and w in FP64, from the FP32 outputs).

    * A pair mass s = (E_i + E_j)^2 - |p_i + p_j|^2 from FP32 components: four sums and three
      fused multiply-adds, each rounding by at most 2^-24 of a term bounded by (E_i + E_j)^2, so
      |ds| <= 8 2^-24 (E_i + E_j)^2.
    * BW(s) = 1/(m0^2 - s - i m0 G) has dBW/ds = BW^2, so |dA| <= |BW_a|^2 |ds12| + |c| |BW_b|^2 |ds23|
      and d|A|^2 <= 2 |A| |dA|; near the phi(1020) (m0 G = 4.1e-3 GeV^2) this is the large term.
    * The rest (m0^2 - s, the reciprocal of |m0^2 - s|^2 + (m0 G)^2 by rcp.approx, the real and
      imaginary parts, their squares) is about a dozen FP32 roundings (rcp.approx: up to 2 ulp)
      of terms no larger than the amplitudes before they interfere; 32 2^-24 (|BW_a| + |c| |BW_b|)^2
      bounds them, also where the two amplitudes cancel and |A|^2 itself is small.
    * The product with w rounds once more: 2^-24 f (2^-23 with the rcp.approx ulp)."""
    m0a, ga, m0b, gb, cabs, carg = params
    c = cabs * np.exp(1j * carg)
    u = 2.0 ** -24
    s, ds = [], []
    for i, j in ((0, 1), (1, 2)):
        v = ev[i] + ev[j]
        s.append(v[0] ** 2 - v[1] ** 2 - v[2] ** 2 - v[3] ** 2)
        ds.append(8 * u * v[0] ** 2)
    bwa = 1.0 / (m0a ** 2 - s[0] - 1j * m0a * ga)
    bwb = 1.0 / (m0b ** 2 - s[1] - 1j * m0b * gb)
    amp = np.abs(bwa + c * bwb)
    f = w * amp ** 2
    return (w * (2 * amp * (np.abs(bwa) ** 2 * ds[0] + cabs * np.abs(bwb) ** 2 * ds[1])
                 + 32 * u * (np.abs(bwa) + cabs * np.abs(bwb)) ** 2) + 2 * u * f)


def test_evaluate_fp32_and_flat():
    """FP32 evaluation on FP32 events against the oracle on the same events: every value within
    its derived per-event bound (fp32_dalitz_value_bound), the sum within 2e-4 relative (the
    bound of the parity module for FP32 sums near the narrow pole)."""
    d = workloads.D0_DALITZ
    nev = 50_001
    gp, gw = hp.generate(d["M"], d["masses"], nev, 2, dtype="f32")
    res, vals = hp.evaluate(gp, gw, me=hp.ME_DALITZ_2BW, params=d["params"], dtype="f32", want_values=True)
    ev64 = gp[:, :, :nev].double().cpu().numpy()
    w64 = gw.double().cpu().numpy()
    ref_vals, ref_sums = oracle.evaluate(ev64, w64, me=1, params=d["params"])
    assert abs(res["sum_f"] - ref_sums[0]) <= 2e-4 * ref_sums[0]
    bound = fp32_dalitz_value_bound(ev64, w64, d["params"])
    err = np.abs(vals.double().cpu().numpy() - ref_vals)
    assert (err <= bound).all(), float((err / bound).max())
    assert float(np.median(bound / ref_vals)) < 1e-4  # the bound is tight where nothing cancels
    flat, fv = hp.evaluate(gp, gw, dtype="f32", want_values=True)
    assert torch.equal(fv, gw)
    assert flat["sum_w"] == flat["sum_f"]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_evaluate_vector_and_scalar_paths_agree(dtype):
    """Aligned events with ld a multiple of the vector width take the 16-byte-load kernel; a
    copy with an odd row stride takes the scalar one.  Same values bit for bit (same per-event
    arithmetic), sums to rounding; ragged tails of both (nevents not a multiple of 2048)."""
    d = workloads.D0_DALITZ
    tdt = torch.float32 if dtype == "f32" else torch.float64
    for nev in (2048 * 3 + 5, 1, 7):
        gp, gw = hp.generate(d["M"], d["masses"], nev, 9, dtype=dtype)
        ld = gp.shape[-1]
        odd = torch.zeros((3, 4, nev + 1 if (nev + 1) % 2 else nev + 2), dtype=tdt, device="cuda")
        odd[:, :, :nev] = gp[:, :, :nev]
        wv = gw[:nev].clone()
        assert ld % 4 == 0 and odd.shape[-1] % 2 == 1
        for me, params in ((hp.ME_DALITZ_2BW, d["params"]), (hp.ME_FLAT, ())):
            rv, vv = hp.evaluate(gp, wv, nev, me=me, params=params, dtype=dtype, want_values=True)
            rs, vs = hp.evaluate(odd, wv, nev, me=me, params=params, dtype=dtype, want_values=True)
            assert torch.equal(vv, vs)
            rtol = 1e-6 if dtype == "f32" else 1e-13
            for k in ("sum_f", "sum_f2", "sum_w", "sum_w2"):
                assert rv[k] == pytest.approx(rs[k], rel=rtol, abs=0.0), k
            assert rv["n"] == rs["n"] == nev


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_sequential_decay_matches_oracle_composition(dtype):
    M, m, sub = 5.0, (0.5, 1.2, 0.3), (0.4, 0.6)
    nev = 4001
    p1, w1, p2, w2 = hp.generate_sequential(M, m, 1, sub, nev, 1, 2, dtype=dtype)
    r1, rw1 = oracle.generate(M, m, nev, seed=1)
    r2, rw2 = oracle.generate_boosted(m[1], sub, nev, seed=2, mothers=r1[1, 1:4, :])
    scale = M
    assert (np.abs(p1[:, :, :nev].double().cpu().numpy() - r1) / scale).max() <= TOL[dtype]
    tol2 = TOL[dtype] if dtype == "f64" else 1e-4  # stage 2 inherits stage 1's FP32 momenta
    assert (np.abs(p2[:, :, :nev].double().cpu().numpy() - r2) / scale).max() <= tol2
    np.testing.assert_allclose((w1 * w2).double().cpu().numpy(), rw1 * rw2, rtol=max(TOL[dtype], 1e-12) * 4)


def test_shutdown_releases_scratch_and_calls_recover():
    """hydra_shutdown frees the scratch of every entry point (integral, evaluation,
    unweighting, VEGAS); later calls allocate again and give the same bits."""
    d = workloads.D0_DALITZ

    def calls():
        r = hp.integrate(d["M"], d["masses"], 1 << 22, 7, me=hp.ME_DALITZ_2BW, params=d["params"])
        p, w = hp.generate(d["M"], d["masses"], 1 << 20, 3, dtype="f64")
        e, _ = hp.evaluate(p, w, me=hp.ME_DALITZ_2BW, params=d["params"], dtype="f64")
        k, _ = hp.unweight(3, w, 3, dtype="f64")
        v = hp.vegas(d["M"], d["masses"], 5, 1 << 24, 2, bins=20, me=hp.ME_DALITZ_2BW, params=d["params"])
        torch.cuda.synchronize()
        return r, e, k.cpu(), v

    def free_after_shutdown():
        hp.shutdown()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return torch.cuda.mem_get_info()[0]

    calls()  # loads every kernel once, so module memory is not counted below
    free0 = free_after_shutdown()
    r1, e1, k1, v1 = calls()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 > 150e6  # VEGAS alone holds 2^24 x 12 bytes of point scratch
    free2 = free_after_shutdown()
    assert free2 >= free0 - 8e6
    r2, e2, k2, v2 = calls()
    assert r1 == r2 and e1 == e2
    assert torch.equal(k1, k2)
    assert np.array_equal(v1["est"], v2["est"]) and np.array_equal(v1["grid"], v2["grid"])


def test_probes_measure_plausible_ceilings():
    """The roofline probes: FP32 FMA rate within the SM issue limit, FP64 far below it, a
    write bandwidth between 1 TB/s and the HBM3e nominal 7.7 TB/s; bad arguments refused."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32 = hp.probe_fma_rate("f32", 20_000)
    f64 = hp.probe_fma_rate("f64", 500)
    assert 0.3 * sms * 128 * 1.0e9 < f32 < sms * 128 * 2.2e9
    assert 0 < f64 < f32 / 8
    buf = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
    gbs = hp.probe_write_bandwidth(buf, 2)
    assert 1000 < gbs < 7700
    with pytest.raises(hp.HydraError, match="MISALIGNED"):
        hp.probe_write_bandwidth(buf[1:], 1)
    with pytest.raises(hp.HydraError, match="INVALID_ARG"):
        hp.probe_fma_rate("f32", 0)


def test_compensated_reduction_against_fsum():
    """The integral's tile / segment reduction (FP64: plain sums inside a 2048-event tile, at
    most ~16 additions deep; Neumaier-compensated across tiles and segments) against
    math.fsum, the correctly rounded sum, of the very per-event values it reduces: 3e7 Dalitz
    f values (about 15 segments) and an adversarial mix of magnitudes 1e-8..1e8 with
    alternating signs.  Bound: 16 roundings of 2^-53 relative to the sum of magnitudes (a
    sequential sum of 3e7 terms can lose ~1e-9)."""
    import math
    d = workloads.D0_DALITZ
    nev = 30_000_001
    p, w = hp.generate(d["M"], d["masses"], nev, 13, dtype="f64")
    res, vals = hp.evaluate(p, w, me=hp.ME_DALITZ_2BW, params=d["params"], dtype="f64", want_values=True)
    v = vals[:nev].cpu().numpy()
    exact = math.fsum(v)
    assert abs(res["sum_f"] - exact) <= 2e-15 * abs(exact), (res["sum_f"], exact)
    exact2 = math.fsum(v * v)
    assert abs(res["sum_f2"] - exact2) <= 2e-15 * abs(exact2)
    # adversarial: weights alternating in sign over 16 decades, flat matrix element (f = w)
    rng = np.random.default_rng(8)
    m = 5_000_003
    ww = rng.uniform(1, 10, m) * 10.0 ** rng.integers(-8, 9, m) * np.where(np.arange(m) % 2, -1.0, 1.0)
    wt = torch.from_numpy(ww).cuda()
    pp = torch.zeros((3, 4, m), dtype=torch.float64, device="cuda")
    r2, _ = hp.evaluate(pp, wt, me=hp.ME_FLAT, dtype="f64")
    exact3 = math.fsum(ww)
    scale = math.fsum(np.abs(ww))
    assert abs(r2["sum_f"] - exact3) <= 2e-15 * scale, (r2["sum_f"], exact3, scale)


@pytest.mark.parametrize("kin", ["f64", "f32"])
def test_dalitz_integrand_closed_form_equals_the_event_construction(kin):
    """The N = 3 Dalitz integral computes E1 from the draws in closed form (no 4-vectors); on
    the same events, the matrix element evaluated from the generator's stored 4-vectors (s_ij
    = (p_i + p_j)^2) gives the same sums: to 1e-12 in FP64, to 2e-5 in FP32."""
    d = workloads.D0_DALITZ
    nev = 1_000_003
    r = hp.integrate(d["M"], d["masses"], nev, 31, kin_dtype=kin, me=hp.ME_DALITZ_2BW, params=d["params"],
                     event_offset=77)
    p, w = hp.generate(d["M"], d["masses"], nev, 31, dtype=kin, event_offset=77)
    e, _ = hp.evaluate(p, w, nevents=nev, me=hp.ME_DALITZ_2BW, params=d["params"], dtype=kin)
    tol = 1e-12 if kin == "f64" else 2e-5
    assert abs(r["sum_f"] - e["sum_f"]) <= tol * abs(e["sum_f"])
    assert abs(r["sum_f2"] - e["sum_f2"]) <= 2 * tol * abs(e["sum_f2"])
    assert abs(r["sum_w"] - e["sum_w"]) <= tol * abs(e["sum_w"])

"""Host logic of the benchmark's roofline bookkeeping (no GPU).

kernel_rooflines turns per-kernel event totals into achieved rates.  Its
algorithmic bytes and flops per unit must be the closed forms for the
20000-triangle workload (T = 20000, r = 3, m = 40, s = 3, binary32 factors,
double-float vectors): operator product 8(r+1)m^2 T + 8 m^2 T + 16 s n =
1.3184 GB; two-colour preconditioner launches 0.8016 GB and 0.4128 GB (level
form 0.6048 GB and 0.6144 GB); stage assembly 2.816 GB; block products
4 s m^3 per lower block (two products of 2 m^3 flops), (nnzb - T)/2 lower
blocks per stage: 23.04 GFLOP; inverses 2 s T m^3 = 7.68 GFLOP.  The roofline object reports the kernel with the largest total
time against the right peak, and the traffic field only when the recorded
source hash matches.
"""
import types

import pytest

import bench


def workload():
    T, m, s, r = 20000, 40, 3, 3
    return types.SimpleNamespace(T=T, m=m, s=s, nnzb=T * (r + 1)), r


def acc_with(times):
    acc = dict(launches=0, iters=[10, 15, 18] * 5, n_matvec=215, n_precond=215, n_ortho=215, ortho_ms=1.0,
               factor_ms=1.0, precond_ms=1.0, matvec_ms=times.get("matvec", 0.0), n_factor=15)
    for k in ("sweep_fwd", "sweep_bwd", "factor_assemble", "factor_products", "factor_inverse"):
        acc[k + "_ms"] = times.get(k, 0.0)
    return acc


@pytest.mark.parametrize("two_colour,fwd,bwd", [(True, 801.6e6, 412.8e6), (False, 604.8e6, 614.4e6)])
def test_algorithmic_amounts(two_colour, fwd, bwd):
    P, r = workload()
    _, k = bench.kernel_rooflines(P, r, acc_with({"matvec": 64.5}), 6783.5, "measured", two_colour=two_colour)
    assert k["matvec"]["alg_bytes"] == pytest.approx(1.3184e9, rel=1e-12)
    assert k["sweep_fwd"]["alg_bytes"] == pytest.approx(fwd, rel=1e-12)
    assert k["sweep_bwd"]["alg_bytes"] == pytest.approx(bwd, rel=1e-12)
    assert k["factor_assemble"]["alg_bytes"] == pytest.approx(2.816e9, rel=1e-12)
    assert k["factor_products"]["alg_flops"] == pytest.approx(23.04e9, rel=1e-12)
    assert k["factor_inverse"]["alg_flops"] == pytest.approx(7.68e9, rel=1e-12)


def test_dominant_kernel_and_rates(monkeypatch):
    P, r = workload()
    monkeypatch.setattr(bench, "traffic_record", lambda name: 1.3378e9 if name == "matvec" else None)
    times = {"matvec": 64.5, "sweep_fwd": 30.1, "sweep_bwd": 18.2, "factor_assemble": 8.1,
             "factor_products": 11.06, "factor_inverse": 14.6}
    roof, k = bench.kernel_rooflines(P, r, acc_with(times), 6783.5, "measured", two_colour=True)
    avg = 64.5 / 215
    assert roof["kernel"] == "matvec" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(1.3184e9 / (avg * 1e6), rel=1e-12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6783.5, rel=1e-12)
    assert roof["traffic"] == 1.3378e9
    # per factorisation: 15 sampled solves, one factorisation each
    assert k["factor_products"]["avg_ms"] == pytest.approx(11.06 / 15, rel=1e-12)
    # a compute-bound kernel on top reports against its own peak
    times2 = dict(times, factor_inverse=1000.0)
    roof2, _ = bench.kernel_rooflines(P, r, acc_with(times2), 6783.5, "measured", two_colour=True)
    assert roof2["kernel"] == "factor_inverse" and roof2["bound"] == "alu" and roof2["unit"] == "TFLOP/s"
    assert roof2["peak"] == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12, rel=1e-12)


def test_traffic_needs_matching_source_hash(tmp_path, monkeypatch):
    """A traffic line counts only while the kernel's source file hashes to the
    recorded value."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = tmp_path / "paper_1701_07181_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_bytes(b"kernel source")
    import hashlib
    h = hashlib.sha256(b"kernel source").hexdigest()[:12]
    (prof / "dram_traffic_c1.txt").write_text("# header\nmatvec 123 k.cu %s\nsweep_fwd 456 k.cu 000000000000\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("matvec") == 123.0
    assert bench.traffic_record("sweep_fwd") is None
    assert bench.traffic_record("factor_inverse") is None

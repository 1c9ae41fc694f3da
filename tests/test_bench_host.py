"""Host-side logic of bench.py (no GPU): the algorithmic work model behind the
roofline fraction, and the parsing of the clock samples that flags throttling."""
import bench


# two-point flux evaluations per element: 3 n^2 n(n-1)/2 volume pairs + 6 n^3 hybrid
# pairs + 3 n^2 face fluxes, tabulated independently of the code for p = 3..7
FLUX_EVALS = {3: 720, 4: 1575, 5: 3024, 6: 5292, 7: 8640}


def test_flux_evaluation_counts():
    for p, total in FLUX_EVALS.items():
        n = p + 1
        _, counts = bench.volume_kernel_flops(1, p)
        assert counts["volume_pairs"] + counts["hybrid"] + 3 * n * n == total


def test_volume_flops_at_p4():
    # 1,500 fluxes x (55 + 20) + face combination 6 n^2 (5 + 10 n) + 5 n^3 + rank-one
    # sweeps 120 n^3, n = 5
    flops, counts = bench.volume_kernel_flops(13824, 4)
    assert counts["flops_per_element"] == 1500 * 75 + 150 * 55 + 625 + 120 * 125 == 136375
    assert flops == 136375 * 13824
    # c = 0: no weight-adjusted sweeps
    _, c0 = bench.volume_kernel_flops(1, 4, has_k=False)
    assert c0["flops_per_element"] == 136375 - 120 * 125


def test_ranocha_flops_at_p4():
    # Ranocha's pressure terms: 1,500 fluxes x (62 + 20), the same face combination, 1/(w J)
    # and sweeps, and 2 flops per node for the pressures; its face fluxes 75 x (62 + 4)
    _, counts = bench.volume_kernel_flops(1, 4, vol_flux="ranocha")
    assert counts["flops_per_element"] == 1500 * 82 + 150 * 55 + 625 + 120 * 125 + 2 * 125 == 147125
    models = bench.stage_kernel_models(4, 1, "fp64", vol_flux="ranocha")
    assert models["volume"] == ("flops", 147125)
    assert models["face_flux"] == ("flops", 75 * 66)
    assert bench.stage_kernel_models(4, 1, "fp64")["face_flux"] == ("flops", 75 * 55)


def test_wa_inverse_flops_at_p4():
    # six rank-one sweeps of 2 n multiply-adds per line (120 n^3 flops per element) and the
    # 1/(W J) scaling (5 n^3), n = 5; without K only the scaling
    e = bench.wa_inverse_roofline({"volume_ms_dudt": 3.0, "volume_ms_raw": 2.0, "ms": 1.0}, 4, 10,
                                  {"sm_mhz": 2000.0}, None)
    assert e["work_per_launch"] == 15625 * 10
    assert abs(e["achieved"] - 15625 * 10 / 1e-3 / 1e12) < 1e-15
    e0 = bench.wa_inverse_roofline({"volume_ms_dudt": 3.0, "volume_ms_raw": 2.0, "ms": 1.0}, 4, 10,
                                   {"sm_mhz": 2000.0}, None, has_k=False)
    assert e0["work_per_launch"] == 625 * 10


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = lines
    return s


def test_clock_samples_report_throttle_reasons():
    ok = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    hot = "0, 1800, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active"
    cap = "0, 1950, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    r = _sampler([ok, ok, ok]).stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    r = _sampler([ok, hot, cap, "garbled"]).stop()
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert r["samples"] == 3 and r["sm_mhz"] == 1950.0


def test_clock_sampler_without_nvidia_smi():
    r = bench.ClockSampler(0).stop()
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


class _Props:
    pci_domain_id, pci_bus_id, pci_device_id = 0, 0x1B, 0


def test_smi_id_is_the_pci_bus_id_when_nvidia_smi_accepts_it(monkeypatch):
    import subprocess
    import torch
    calls = []

    def fake_run(cmd, **kw):
        calls.append(cmd)
        return subprocess.CompletedProcess(cmd, 0, stdout="3\n", stderr="")

    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: _Props())
    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    bench.smi_id.cache_clear()
    assert bench.smi_id(0) == "00000000:1B:00.0"
    assert calls[0][1] == "--id=00000000:1B:00.0"
    # refused by nvidia-smi, or no bus id: the CUDA ordinal
    monkeypatch.setattr(bench.subprocess, "run",
                        lambda cmd, **kw: subprocess.CompletedProcess(cmd, 6, stdout="", stderr="no"))
    bench.smi_id.cache_clear()
    assert bench.smi_id(1) == "1"

    def no_props(d):
        raise RuntimeError("no CUDA")

    monkeypatch.setattr(torch.cuda, "get_device_properties", no_props)
    bench.smi_id.cache_clear()
    assert bench.smi_id(2) == "2"
    bench.smi_id.cache_clear()


def test_cpu_baseline_times_the_oracle_on_one_and_on_several_workers():
    val, med, stages = bench._pool_run(2, 2, 0.5, 1)
    assert val > 0 and med > 0 and stages >= 1
    val2, med2, stages2 = bench._pool_run(2, 2, 0.5, 2)
    assert val2 > 0 and stages2 >= 2
    info = bench.host_info()
    assert info["nproc"] >= 1

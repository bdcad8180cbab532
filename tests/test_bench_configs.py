"""Host logic of bench.py, on the CPU: every benchmark workload lowers to the
kernels its schedules name, at its full size (the fused and stage-per-kernel
schedules, and the dominant group timed alone where a step has several); the
clocks record summarises the samples of the timed region."""

import importlib.util
import os

import pytest

import __graft_entry__
from paper_2012_07145_gb300 import hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def table():
    __graft_entry__.build()
    spec = importlib.util.spec_from_file_location("bench_cfg", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b.config_table()


def _sizes(inputs):
    return [(a.shape[-1], a.shape[-2]) for a, _ in inputs]


def test_every_workload_lowers(table):
    assert {"chain32", "harris", "unsharp", "histeq", "ll", "maxfilter", "interpolate", "bilateral"} <= set(table)
    for name, cfg in table.items():
        sizes = [(cfg["w"], cfg["h"])]
        plain = cfg["build"]()
        fused = cfg["build"]()
        cfg["fused"](fused)
        for p in (plain, fused):
            kinds = [p.group_info(sizes, g).kernel for g in range(p.group_count())]
            assert all(0 <= k < len(hp.KERNEL_NAMES) for k in kinds), name
        if "dominant" in cfg:
            dom = cfg["dominant"]
            d = dom["build"]()
            dsizes = _sizes(dom["inputs"](0)) if "inputs" in dom else sizes
            assert d.group_count() == 1
            assert hp.KERNEL_NAMES[d.group_info(dsizes, 0).kernel] == dom["kernel"][2:], name


def test_fused_schedules_use_the_specialised_kernels(table):
    expect = {"chain32": "stencil_chain", "harris": "harris_rows", "unsharp": "stencil_rows", "histeq": "histeq",
              "maxfilter": "max_rows", "bilateral": "grid_blur", "interpolate": "interp_rows", "ll": "ll_remap_rows"}
    for name, kname in expect.items():
        cfg = table[name]
        p = cfg["build"]()
        cfg["fused"](p)
        names = [hp.KERNEL_NAMES[p.group_info([(cfg["w"], cfg["h"])], g).kernel] for g in range(p.group_count())]
        assert kname in names, (name, names)
        assert "generic" not in names, (name, names)   # no group falls back to the interpreter


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_clk", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary_takes_the_timed_region_and_names_throttle_reasons():
    """The clocks record of a bench line: the median SM clock of the samples
    inside the timed region, the maximum clock, and every throttle reason seen
    active there (samples before or after the region are ignored)."""
    b = _bench_module()
    c = b.ClockSampler(0)
    c.proc = _DoneProcess()
    row = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"
    c.lines = [(0.0, row.format(sm=1000, hw="Active", pc="Not Active")),        # before the region
               (1.0, row.format(sm=2070, hw="Not Active", pc="Not Active")),
               (1.1, row.format(sm=1980, hw="Not Active", pc="Active")),
               (1.2, row.format(sm=2070, hw="Not Active", pc="Not Active")),
               (1.3, "garbage line"),
               (9.0, row.format(sm=500, hw="Active", pc="Not Active"))]         # after the region
    c.t0, c.t1 = 0.9, 1.25
    out = b.ClockSampler.stop(c)
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines.append((1.15, row.format(sm=1400, hw="Active", pc="Not Active")))
    out = b.ClockSampler.stop(c)
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"] and out["samples"] == 4


def test_clock_summary_of_a_region_shorter_than_the_sampling_period():
    b = _bench_module()
    c = b.ClockSampler(0)
    c.proc = _DoneProcess()
    c.lines = [(0.0, "0, 1500, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"),
               (2.0, "0, 2070, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active")]
    c.t0, c.t1 = 1.0, 1.01           # no sample inside: the first one after the region starts
    assert b.ClockSampler.stop(c)["sm_mhz"] == 2070.0


@pytest.mark.parametrize("size", [(1, 1), (2, 3), (7, 5), (33, 17), (250, 130)])
def test_every_workload_lowers_at_tiny_and_ragged_sizes(table, size):
    """Degenerate and ragged images lower under both schedules of every
    workload (a pyramid of 1x1 levels, one partial tile or strip)."""
    for name, cfg in table.items():
        plain = cfg["build"]()
        fused = cfg["build"]()
        cfg["fused"](fused)
        for p in (plain, fused):
            for g in range(p.group_count()):
                info = p.group_info([size], g)
                assert 0 <= info.kernel < len(hp.KERNEL_NAMES), (name, size, g)
                assert info.grid_x >= 1 and info.grid_y >= 1 and info.threads >= 32, (name, size, g)


def test_chain_flop_counts_are_the_methods_work(table):
    """The ALU roofline counts the method's work: 14 flops per binomial stage
    and 10 per box stage (a separable pass: ((a+e) + 4(b+d)) + 6c then x 1/16,
    or (((a+b) + (c+d)) + e) x 1/5; an fma counts 2), not the kernel's own
    instruction mix, which is reported separately as FP32 instructions."""
    assert table["chain32"]["flops_px"] == 16 * 14 + 16 * 10 == 384
    assert table["chain4"]["flops_px"] == 4 * 14 == 56
    assert table["chain32"]["fp32_instr_px"] == 320
    names = set(table) | {"serving"}
    spec = importlib.util.spec_from_file_location("bench_cfg2", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert set(b.DEFAULT_CONFIGS.split(",")) <= names

"""Every benchmark workload lowers, on the CPU, to the kernels its schedules
name, at its full size (no GPU needed): the fused and stage-per-kernel
schedules, and the dominant group timed alone where a step has several."""

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

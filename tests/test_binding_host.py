"""Host-side marshalling of the Python binding (no GPU): mb_opts defaults,
name-to-enum mappings and the per-launch time limit default."""
import pytest

import paper_2007_00745_gb300 as mb


def test_opts_defaults_are_the_c_defaults():
    o = mb._opts(stream=1)
    assert o.sched == mb.MB_SCHED_FCFS_TILES and o.tile == 0 and o.grid == 0 and o.block == 0 and o.unroll == 0
    assert o.precision == mb.MB_PREC_FP64 and o.cycle_check == 0 and o.fp64_products == 0
    assert o.split == 0 and o.round_tiles == 0 and o.stream == 1
    assert not o.items and not o.trace and not o.status and not o.workspace


def test_opts_names_map_to_enums():
    for name, val in mb.SCHEDS.items():
        assert mb._opts(stream=1, sched=name).sched == val
    for name, val in mb.PRECISIONS.items():
        assert mb._opts(stream=1, precision=name).precision == val
    assert mb._opts(stream=1, precision=2).precision == mb.MB_PREC_DFLOAT
    with pytest.raises(KeyError):
        mb._opts(stream=1, precision="fp16")
    with pytest.raises(KeyError):
        mb._opts(stream=1, sched="round_robin")


def test_time_limit_default(monkeypatch):
    monkeypatch.setattr(mb, "DEFAULT_MAX_SECONDS", 0)
    assert mb._opts(stream=1).max_seconds == 0           # the C API's default: no limit
    monkeypatch.setattr(mb, "DEFAULT_MAX_SECONDS", 42)
    assert mb._opts(stream=1).max_seconds == 42
    assert mb._opts(stream=1, max_seconds=5).max_seconds == 5

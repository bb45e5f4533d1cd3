"""Launch-shape tuning, host side (no GPU): the committed table of
sg_autotune results parses, every choice is in the range sg_tune_set
accepts, lookups find the benchmark sizes, malformed tables are refused,
and the C ABI validates its arguments before touching a device."""
import ctypes as C
import json
import os

import pytest

from paper_2209_14740_gb300 import tune_table


def test_committed_table_is_valid_and_covers_the_workloads():
    assert os.path.exists(tune_table.TABLE_PATH), "tune_table.json is committed beside tune_table.py"
    tab = tune_table.load_table()
    with open(tune_table.TABLE_PATH) as fh:
        doc = json.load(fh)
    assert len(tab) == len(doc["entries"]) >= 3
    for e in doc["entries"]:
        assert e["cgs_us"] > 0 and e["op_us"] > 0
        assert (e["apply_us"] > 0) == (e["tc_tile_n"] in (64, 128, 256))
    # the headline, the 127^2 and the 1D workloads have entries
    assert tune_table.lookup(2, 511, 511, 6, 3) is not None
    assert tune_table.lookup(2, 127, 127, 3, 3) is not None
    assert tune_table.lookup(1, 200, 1, 1, 5) is not None
    assert tune_table.lookup(2, 12345, 3, 1, 1) is None


@pytest.mark.parametrize("bad", [{"cgs_blocks_per_sm": 9}, {"op_ctas_per_sm": -1}, {"tc_tile_n": 96}])
def test_out_of_range_choice_is_refused(tmp_path, bad):
    e = {"dim": 2, "mx": 31, "my": 31, "s": 2, "r": 2, "cgs_blocks_per_sm": 3, "op_ctas_per_sm": 1, "tc_tile_n": 64}
    e.update(bad)
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"entries": [e]}))
    with pytest.raises(ValueError):
        tune_table.load_table(str(p))


def test_duplicate_size_is_refused(tmp_path):
    e = {"dim": 2, "mx": 31, "my": 31, "s": 2, "r": 2, "cgs_blocks_per_sm": 3, "op_ctas_per_sm": 1, "tc_tile_n": 64}
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"entries": [e, dict(e, cgs_blocks_per_sm=4)]}))
    with pytest.raises(ValueError):
        tune_table.load_table(str(p))


def test_abi_struct_and_argument_checks_without_gpu():
    from paper_2209_14740_gb300 import binding
    lib = binding.load()
    assert C.sizeof(binding.SgTune) == 4 * 4 + 3 * 8
    t = binding.SgTune()
    assert lib.sg_tune_get(None, C.byref(t)) == binding.SG_EINVAL
    assert lib.sg_tune_set(None, C.byref(t)) == binding.SG_EINVAL
    assert lib.sg_autotune(None, 30, C.byref(t), None) == binding.SG_EINVAL

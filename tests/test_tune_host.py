"""The batch tuning table's file format (host only, no GPU): a written table reads back unchanged, a file
that is not such a table is refused and changes nothing."""
import json

import pytest

from paper_2511_14664_gb300 import qsim


def test_tuning_file_round_trip(tmp_path):
    src = tmp_path / "in.json"
    src.write_text(json.dumps({"format": "qsim-batch-tune-1", "k_by_width": {"10": 3, "14": 4, "21": 2},
                               "tc_min_n": {"1": 22, "3": 18}}))
    qsim.batch_tune_load(str(src))
    out = tmp_path / "out.json"
    qsim.batch_tune_save(str(out))
    d = json.loads(out.read_text())
    assert d["format"] == "qsim-batch-tune-1"
    assert {k: d["k_by_width"][k] for k in ("10", "14", "21")} == {"10": 3, "14": 4, "21": 2}
    assert d["tc_min_n"]["1"] == 22 and d["tc_min_n"]["3"] == 18
    qsim.batch_tune_load(str(out))          # what it writes, it reads


@pytest.mark.parametrize("text", [
    "not json at all",
    '{"format": "qsim-batch-tune-1", "k_by_width": {"10": 9}, "tc_min_n": {}}',    # k beyond 4
    '{"format": "qsim-batch-tune-1", "k_by_width": {}, "tc_min_n": {"1": 40}}',    # threshold beyond 27
    '{"format": "other", "k_by_width": {}, "tc_min_n": {}}',
])
def test_bad_tuning_files_are_refused(tmp_path, text):
    good = tmp_path / "good.json"
    good.write_text(json.dumps({"format": "qsim-batch-tune-1", "k_by_width": {"11": 2}, "tc_min_n": {"2": 24}}))
    qsim.batch_tune_load(str(good))
    bad = tmp_path / "bad.json"
    bad.write_text(text)
    with pytest.raises(qsim.QsimError) as e:
        qsim.batch_tune_load(str(bad))
    assert e.value.code == 1
    out = tmp_path / "out.json"
    qsim.batch_tune_save(str(out))
    d = json.loads(out.read_text())
    assert d["k_by_width"]["11"] == 2 and d["tc_min_n"]["2"] == 24   # unchanged by the refused file


def test_missing_file_is_refused(tmp_path):
    with pytest.raises(qsim.QsimError):
        qsim.batch_tune_load(str(tmp_path / "absent.json"))

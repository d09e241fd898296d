"""The committed ncu records of the fused step are tied to its code by a hash
of the kernel sources without comments or whitespace (bench.py): a record is
used only while the code it was taken on is unchanged."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_code_tokens_drop_comments_and_whitespace_only():
    a = 'int a = 1;  // note\n/* block\n comment */ const char *s = "x // y /* z */";\nchar q = \'"\';'
    b = 'int a=1;\n\n   const char *s="x // y /* z */"; char q=\'"\';   // other note'
    assert bench._code_tokens(a) == bench._code_tokens(b)
    # string and character literals are code: a change inside one counts
    assert bench._code_tokens(a) != bench._code_tokens(a.replace('"x // y', '"x / y'))
    # so does any change of the code itself
    assert bench._code_tokens(a) != bench._code_tokens(a.replace("a = 1", "a = 2"))


def test_records_are_used_only_for_the_code_they_were_taken_on(monkeypatch):
    with open(os.path.join(ROOT, "profiles", "smo_step_covtype_fp64_traffic.json")) as fh:
        taken_on = json.load(fh)["kernel_source_hash"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda root=ROOT: taken_on)
    assert bench.measured_traffic("covtype", "fp64") is not None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda root=ROOT: "0" * 16)
    assert bench.measured_traffic("covtype", "fp64") is None
    assert bench.measured_issue("covtype", "fp64") is None

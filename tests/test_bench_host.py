"""Host logic of bench.py: the counters recorded from ncu are tied to the counting kernel's
code, not to the wording of its comments."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_drops_comments_and_keeps_code():
    src = 'int a = 1; // one\n/* block\n comment */ const char *s = "x // y";\n'
    assert bench._code_only(src) == 'int a = 1; const char *s = "x // y";'
    reworded = src.replace("// one", "// the first").replace("block", "other words")
    assert bench._code_only(reworded) == bench._code_only(src)
    assert bench._code_only(src.replace("a = 1", "a = 2")) != bench._code_only(src)


def test_kernel_hash_follows_code_changes_only():
    text = {n: open(os.path.join(ROOT, "paper_2605_14743_gb300", "csrc", n)).read()
            for n in bench.KERNEL_SOURCES}
    base = bench.kernel_source_hash(lambda n: text[n])
    assert base == bench.kernel_source_hash()
    name = bench.KERNEL_SOURCES[1]
    commented = dict(text, **{name: "// a new comment line\n" + text[name]})
    assert bench.kernel_source_hash(lambda n: commented[n]) == base
    changed = dict(text, **{name: text[name] + "\nstatic const int kProbe = 1;\n"})
    assert bench.kernel_source_hash(lambda n: changed[n]) != base


def test_recorded_counters_file_has_its_fields():
    fields = {}
    with open(bench.TRAFFIC_FILE) as f:
        for line in f:
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                fields[k] = v
    for k in ("source_sha256", "realizations_per_launch", "dram_bytes_read", "dram_bytes_write",
              "warp_instructions_per_realization"):
        assert k in fields
    assert len(fields["source_sha256"]) == 64

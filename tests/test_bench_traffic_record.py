"""The bench's traffic record on CPU: a profile summary's `traffic_record:` line gives the DRAM
bytes of a step's kernel only while the kernel's sources hash as they did at capture time, so a
changed kernel reports null traffic instead of a stale figure."""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _setup(tmp_path, a=b"kernel a\n", b=b"header b\n"):
    src = tmp_path / "src"
    prof = tmp_path / "profiles"
    src.mkdir()
    prof.mkdir()
    (src / "k.cu").write_bytes(a)
    (src / "k.cuh").write_bytes(b)
    digest = hashlib.sha256(a + b).hexdigest()
    (prof / "k_c3.md").write_text("# summary\n\ntraffic_record: jacobi | k_x | k.cu+k.cuh | %s | 12345\n" % digest)
    return str(prof), str(src)


def test_record_holds_while_the_sources_match(tmp_path):
    prof, src = _setup(tmp_path)
    assert bench.traffic_record("jacobi", prof, src) == 12345.0
    assert bench.traffic_record("core", prof, src) is None   # no record for that step


def test_record_lapses_when_a_source_changes_or_goes(tmp_path):
    prof, src = _setup(tmp_path)
    with open(os.path.join(src, "k.cuh"), "ab") as f:
        f.write(b"// edited\n")
    assert bench.traffic_record("jacobi", prof, src) is None
    os.remove(os.path.join(src, "k.cu"))
    assert bench.traffic_record("jacobi", prof, src) is None

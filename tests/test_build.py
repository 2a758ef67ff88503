"""The in-tree build rebuilds an object when any header it may include is
newer than the object (a regenerated noise table must not leave a library
compiled from the old one).  No GPU needed."""
import os

from paper_2002_03120_gb300 import build


def test_header_edit_marks_objects_stale(tmp_path):
    src = os.path.join(build.CSRC, "k_pairs.cu")
    obj = tmp_path / "k_pairs.o"
    obj.write_bytes(b"")
    newest = max(os.path.getmtime(p) for p in [src] + build.headers())
    os.utime(obj, (newest + 10, newest + 10))
    assert not build._stale(str(obj), src)
    tables = os.path.join(build.CSRC, "bm_tables.cuh")
    assert tables in build.headers()
    os.utime(obj, (os.path.getmtime(tables) - 10, os.path.getmtime(tables) - 10))
    assert build._stale(str(obj), src)
    assert build._stale(str(tmp_path / "missing.o"), src)

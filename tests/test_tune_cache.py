"""The autotuner's cache file (st_autotune_save / st_autotune_load) through the C ABI, on the CPU.

Both calls are host-only: entries go through the process-wide table without any CUDA call, so the library is loaded
and exercised here without a GPU.  A cache is applied only on a device with the same tag, implausible entries are
skipped, and a malformed file loads nothing.
"""

import ctypes as C

import pytest

import paper_1912_10082_gb300 as st

TAG = b"NVIDIA GB300 sm_103 152SM"


@pytest.fixture(scope="module")
def L():
    from paper_1912_10082_gb300.build import build

    build()
    return st.lib()


@pytest.fixture(autouse=True)
def empty_table(L):
    L.st_autotune_reset()
    yield
    L.st_autotune_reset()


def load(L, path, tag=TAG):
    n = C.c_int(-1)
    rc = L.st_autotune_load(str(path).encode(), tag, C.byref(n))
    return rc, n.value


ENTRIES = ["1 8 0 255 255 2 1", "1 8 1 255 255 4 2", "2 4 255 508 2 0 0", "1 4 1 63 3969 126 0"]


def write_cache(path, tag=TAG.decode(), rows=ENTRIES, header="st-autotune 1"):
    path.write_text("\n".join([header, f"device {tag}"] + list(rows)) + "\n")


def test_load_save_round_trip(L, tmp_path):
    src = tmp_path / "a.txt"
    write_cache(src, rows=ENTRIES[::-1] + [""])   # unsorted, with a blank line
    assert load(L, src) == (st.ST_OK, 4)
    assert L.st_autotune_count() == 4
    out = tmp_path / "b.txt"
    assert L.st_autotune_save(str(out).encode(), TAG) == st.ST_OK
    lines = out.read_text().splitlines()
    assert lines[:2] == ["st-autotune 1", "device " + TAG.decode()]
    body = [tuple(int(x) for x in ln.split()) for ln in lines[2:]]
    assert body == sorted(tuple(int(x) for x in e.split()) for e in ENTRIES)
    L.st_autotune_reset()
    assert L.st_autotune_count() == 0
    assert load(L, out) == (st.ST_OK, 4)
    assert L.st_autotune_count() == 4


def test_other_device_loads_nothing(L, tmp_path):
    src = tmp_path / "a.txt"
    write_cache(src)
    assert load(L, src, b"NVIDIA B200 sm_100 148SM") == (st.ST_OK, 0)
    assert L.st_autotune_count() == 0


def test_implausible_entries_are_skipped(L, tmp_path):
    src = tmp_path / "a.txt"
    rows = ENTRIES[:2] + ["3 8 0 1 1 1 0",    # unknown family
                          "1 2 0 1 1 1 0",    # element size 2
                          "1 8 0 1 1 1 3",    # variant index out of range
                          "2 8 5 10 1 0 -1"]  # negative variant
    write_cache(src, rows=rows)
    assert load(L, src) == (st.ST_OK, 2)
    assert L.st_autotune_count() == 2


def test_same_shape_is_replaced(L, tmp_path):
    a, b = tmp_path / "a.txt", tmp_path / "b.txt"
    write_cache(a, rows=["1 8 0 255 255 2 1"])
    write_cache(b, rows=["1 8 0 255 255 2 2"])
    assert load(L, a)[1] == 1 and load(L, b)[1] == 1
    assert L.st_autotune_count() == 1
    out = tmp_path / "c.txt"
    assert L.st_autotune_save(str(out).encode(), TAG) == st.ST_OK
    assert out.read_text().splitlines()[2] == "1 8 0 255 255 2 2"


@pytest.mark.parametrize("rows,header", [(["1 8 0 255 255 2"], "st-autotune 1"),          # six fields
                                         (["1 8 0 255 255 2 1 9"], "st-autotune 1"),      # eight fields
                                         (["1 8 0 255 x 2 1"], "st-autotune 1"),          # not a number
                                         (ENTRIES, "st-autotune 2")])                     # unknown version
def test_malformed_file_loads_nothing(L, tmp_path, rows, header):
    src = tmp_path / "a.txt"
    write_cache(src, rows=list(ENTRIES[:2]) + rows if header == "st-autotune 1" else rows, header=header)
    rc, n = load(L, src)
    assert rc == st.ST_EINVAL and n == 0
    assert L.st_autotune_count() == 0


def test_bad_arguments(L, tmp_path):
    src = tmp_path / "a.txt"
    write_cache(src)
    assert load(L, src, b"") == (st.ST_EINVAL, 0)
    assert load(L, src, b"two\nlines") == (st.ST_EINVAL, 0)
    assert load(L, src, b"x" * 200) == (st.ST_EINVAL, 0)
    assert load(L, tmp_path / "missing.txt") == (st.ST_EINVAL, 0)
    assert L.st_autotune_save(str(tmp_path / "no_dir" / "c.txt").encode(), TAG) == st.ST_EINVAL
    assert L.st_autotune_save(None, TAG) == st.ST_EINVAL
    assert L.st_autotune_count() == 0

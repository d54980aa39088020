"""The C ABI library: builds for sm_103a, loads, exports every declared entry
point, and validates arguments on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1407_1507_gb300 import build as kbuild
from paper_1407_1507_gb300 import kmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    """Function names declared in include/*.h (extern "C" entry points)."""
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(kmc_\w+)\s*\(", src, flags=re.M):
            names.add(mt.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return kmc.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"kmc_open", "kmc_add_reads", "kmc_count", "kmc_result", "kmc_close"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", kbuild.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = sorted(n for n in names if n not in exported)
    assert not missing, f"declared but not exported: {missing}"
    for n in names:
        assert hasattr(lib, n)
    # the binding declares exactly the exported C names
    assert {s[0] for s in kmc.SIGNATURES} == names


def test_build_targets_sm103a_only():
    assert kbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_default_params_are_the_papers(lib):
    p = kmc.kmc_default_params()
    assert (p.k, p.m, p.n_bins, p.x, p.cutoff_min, p.cutoff_max, p.canonical) == \
        (25, 7, 512, kmc.KMC_AUTO, 2, 10**9, 1)


def test_strerror_names_every_code(lib):
    for code in range(0, -11, -1):
        s = kmc.strerror(code)
        assert s and s != "unknown error"


@pytest.mark.parametrize("field,value", [("k", 0), ("k", 65), ("m", 0), ("m", 12), ("n_bins", 0),
                                         ("n_bins", 65537), ("x", 4), ("canonical", 2),
                                         ("reserved0", 1), ("debug_flags", 64)])
def test_open_rejects_bad_params_on_host(lib, field, value):
    p = kmc.kmc_default_params()
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lib.kmc_open(ctypes.byref(h), ctypes.byref(p)) == kmc.KMC_EINVAL
    assert h.value is None


def test_open_rejects_noncanonical_kx_mers(lib):
    # k-mers as read (Suppl. S1 -b) are counted with x = 0 only
    p = kmc.kmc_default_params()
    p.canonical, p.x = 0, 2
    h = ctypes.c_void_p()
    assert lib.kmc_open(ctypes.byref(h), ctypes.byref(p)) == kmc.KMC_EINVAL


def test_open_rejects_inverted_cutoffs(lib):
    p = kmc.kmc_default_params()
    p.cutoff_min, p.cutoff_max = 5, 4
    h = ctypes.c_void_p()
    assert lib.kmc_open(ctypes.byref(h), ctypes.byref(p)) == kmc.KMC_EINVAL


def test_null_handles_are_rejected(lib):
    n = ctypes.c_uint64()
    assert lib.kmc_count(None) == kmc.KMC_EINVAL
    assert lib.kmc_result_size(None, ctypes.byref(n)) == kmc.KMC_EINVAL
    lib.kmc_close(None)  # no-op
    assert lib.kmc_add_file_bytes(None, b"@a\nA\n+\nI\n", 8, kmc.KMC_FORMAT_FASTQ) == kmc.KMC_EINVAL
    assert lib.kmc_add_file_bytes_device(None, None, 8, kmc.KMC_FORMAT_FASTA) == kmc.KMC_EINVAL
    assert lib.kmc_db_write(None, b"x") == kmc.KMC_EINVAL
    info = kmc.kmc_db_info()
    assert lib.kmc_db_info_get(None, ctypes.byref(info)) == kmc.KMC_EINVAL
    assert lib.kmc_db_lookup(None, None, 1, None, None) == kmc.KMC_EINVAL
    lib.kmc_db_close(None)  # no-op


def test_db_open_rejects_missing_and_malformed_files(lib, tmp_path):
    """The reader checks the format section's markers, header position and
    sizes before touching a device, so malformed files fail on the host."""
    from oracle import kmc_db as DB
    from oracle import strings as S
    reads = ["ACGTTGCAACGGTTACGATCGATCGGATCCA", "TTGCAACGGTTACGATCGAT"]
    cnt = S.count_brute(reads, 12, 1)
    pre, suf = DB.write(12, 5, [S.value(x) for x in cnt], list(cnt.values()), [0] * (4 ** 5 + 1), 1, 1, 10 ** 9)
    db = ctypes.c_void_p()

    def open_with(p_bytes, s_bytes, name):
        base = str(tmp_path / name)
        if p_bytes is not None:
            open(base + ".kmc_pre", "wb").write(p_bytes)
        if s_bytes is not None:
            open(base + ".kmc_suf", "wb").write(s_bytes)
        return lib.kmc_db_open(ctypes.byref(db), os.fsencode(base), 0)

    assert open_with(None, None, "missing") == kmc.KMC_EIO
    assert open_with(pre, None, "no_suffix_file") == kmc.KMC_EIO
    assert open_with(b"KMCX" + pre[4:], suf, "bad_marker") == kmc.KMC_EIO
    assert open_with(pre[:-4] + b"KMCX", suf, "bad_end_marker") == kmc.KMC_EIO
    assert open_with(pre, suf[:-5] + b"KMCS", "truncated_records") == kmc.KMC_EIO
    bad_pos = pre[:-8] + (70).to_bytes(4, "little") + b"KMCP"
    assert open_with(bad_pos, suf, "bad_header_position") == kmc.KMC_EIO
    assert db.value is None
    assert lib.kmc_db_open(None, b"x", 0) == kmc.KMC_EINVAL
    assert "kmc_pre" in kmc.strerror(kmc.KMC_EIO) or "kmc_suf" in kmc.strerror(kmc.KMC_EIO)

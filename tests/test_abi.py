"""The C-ABI library builds, loads and exports every entry point include/cfust.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np

from paper_2005_06848_gb300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(cfust_\w+)\s*\(", text, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("cfust_create", "cfust_destroy", "cfust_loglik", "cfust_estep", "cfust_mstep",
                 "cfust_fit", "cfust_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_rejects_bad_lattice_without_a_device():
    lib = binding.load()
    z = np.array([1, 3, 5], dtype=np.int64)
    sh = np.array([0.1, 0.2, 0.3])
    for n, dim, prec in [(100, 3, 1), (16, 3, 1), (1024, 9, 1), (1024, 3, 7)]:
        lat = binding.cfust_lattice(n, dim, z.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        opts = binding.cfust_opts(prec, lat, 0, 0.0, 0.0, 5, 0.0, 1, 0, 0, 0)
        h = ctypes.c_void_p()
        st = lib.cfust_create(ctypes.byref(h), ctypes.byref(opts), None)
        assert st == -1, (n, dim, prec, st)
        assert lib.cfust_last_error(None)
    bad_shift = np.array([0.1, 1.5, 0.3])
    lat = binding.cfust_lattice(1024, 3, z.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                bad_shift.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    opts = binding.cfust_opts(1, lat, 0, 0.0, 0.0, 5, 0.0, 1, 0, 0, 0)
    h = ctypes.c_void_p()
    st = lib.cfust_create(ctypes.byref(h), ctypes.byref(opts), None)
    assert st in (-1, -6)   # -6 when no device is visible (checked first on some hosts)
    good = binding.cfust_lattice(1024, 3, z.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    for nats in (0.5, -1.0, 701.0, float("nan")):
        opts = binding.cfust_opts(1, good, 0, 0.0, 0.0, 5, 0.0, 1, 0, 0, 0, nats)
        st = lib.cfust_create(ctypes.byref(h), ctypes.byref(opts), None)
        assert st == -1 and b"triage_nats" in lib.cfust_last_error(None), nats


def test_unpack_e4_round_trip():
    r, n = 3, 5
    rng = np.random.default_rng(0)
    A = rng.standard_normal((2, n, r, r))
    A = A + np.swapaxes(A, -1, -2)
    packed = np.stack([A[:, :, t, h] for t in range(r) for h in range(t + 1)], axis=1)  # [2, rp, n]
    assert np.allclose(binding.unpack_e4(packed, r), A)


def test_lattice_spec_is_deterministic():
    a = synth.make_lattice(2048, 4, 3)
    b = synth.make_lattice(2048, 4, 3)
    assert np.array_equal(a.z, b.z) and np.array_equal(a.shift, b.shift)
    assert a.z[0] == 1 and np.all((a.z > 0) & (a.z < 2048))
    assert np.all((a.shift >= 0) & (a.shift < 1))


def test_surrogate_create_rejects_bad_lattice_without_a_device():
    lib = binding.load()
    z = np.array([1, 3, 5], dtype=np.int64)
    sh = np.array([0.1, 0.2, 0.3])
    lat = binding.cfust_lattice(1024, 3, z.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    h = ctypes.c_void_p()
    assert lib.cfust_surrogate_create(ctypes.byref(h), 1, ctypes.byref(lat), None) == -1
    assert b"dim 4" in lib.cfust_surrogate_last_error(None)
    assert lib.cfust_surrogate_create(ctypes.byref(h), 1, None, None) == -1


def test_ctypes_structs_match_the_c_header_layout(tmp_path):
    """The binding's ctypes mirrors of cfust_params, cfust_lattice and
    cfust_opts have the C header's size and field offsets (a field added on
    one side only would shift every later option silently)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("no C compiler")
    structs = {"cfust_params": binding.cfust_params, "cfust_lattice": binding.cfust_lattice,
               "cfust_opts": binding.cfust_opts}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "cfust.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", include, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            parts = line.split()
            got[tuple(parts[:-1])] = int(parts[-1])
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)

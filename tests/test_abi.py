"""The C ABI library builds, loads and exports every declared entry point
(no compute call: these run without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2406_11185_gb300 import adft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "adft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(adft_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(adft.LIB_PATH):
        from paper_2406_11185_gb300 import build
        build.build()
    return adft.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "adft_jk_build" in names and "adft_basis_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(adft.EXPORTED) == sorted(names)


def test_status_strings_and_version(lib):
    assert adft.status_string(0) == "ok"
    assert "symmetric" in adft.status_string(adft.ADFT_ERR_ASYM_D)
    assert lib.adft_version().decode().startswith("adft")


def test_null_arguments_rejected_without_gpu(lib):
    out = ctypes.c_void_p()
    assert lib.adft_basis_create(None, 0, None, 0, 1, ctypes.byref(out)) == adft.ADFT_ERR_ARG
    assert lib.adft_basis_create(None, 0, None, 0, 1, None) == adft.ADFT_ERR_ARG
    assert lib.adft_jk_build(None, None, None, None, None) == adft.ADFT_ERR_ARG
    n = ctypes.c_int()
    assert lib.adft_basis_nbf(None, ctypes.byref(n)) == adft.ADFT_ERR_ARG
    assert len(adft.last_error()) > 0


def _shell_args(shells):
    """ctypes adft_shell array for [(atom, l, exps, coefs)] (arrays kept alive in the result)."""
    keep = []
    arr = (adft.adft_shell * len(shells))()
    for i, (atom, l, exps, coefs) in enumerate(shells):
        e = (ctypes.c_double * len(exps))(*exps)
        c = (ctypes.c_double * len(coefs))(*coefs)
        keep += [e, c]
        arr[i].atom, arr[i].l, arr[i].nprim = atom, l, len(exps)
        arr[i].exps = ctypes.cast(e, ctypes.POINTER(ctypes.c_double))
        arr[i].coefs = ctypes.cast(c, ctypes.POINTER(ctypes.c_double))
    return arr, keep


@pytest.mark.parametrize("bad", ["l_too_high", "too_many_prims", "zero_prims", "bad_exponent", "bad_atom",
                                 "nan_coordinate", "bad_spherical"])
def test_invalid_basis_rejected_before_any_device_work(lib, bad):
    """Every argument error of adft_basis_create is caught on the host, before
    the first CUDA call, so these run without a GPU."""
    xyz = [0.0, 0.0, 0.0, 0.0, 0.0, 1.4]
    shells = [(0, 0, [3.0, 0.5], [0.4, 0.7]), (1, 1, [1.1], [1.0])]
    spherical = 1
    if bad == "l_too_high":
        shells[1] = (1, adft.ADFT_LMAX + 1, [1.1], [1.0])
    elif bad == "too_many_prims":
        n = adft.ADFT_MAX_NPRIM + 1
        shells[0] = (0, 0, [0.1 * 1.5 ** k for k in range(n)], [1.0] * n)
    elif bad == "zero_prims":
        shells[0] = (0, 0, [], [])
    elif bad == "bad_exponent":
        shells[0] = (0, 0, [3.0, -0.5], [0.4, 0.7])
    elif bad == "bad_atom":
        shells[1] = (2, 1, [1.1], [1.0])
    elif bad == "nan_coordinate":
        xyz[4] = float("nan")
    elif bad == "bad_spherical":
        spherical = 2
    arr, keep = _shell_args(shells)
    cxyz = (ctypes.c_double * len(xyz))(*xyz)
    out = ctypes.c_void_p()
    st = lib.adft_basis_create(cxyz, 2, arr, len(shells), spherical, ctypes.byref(out))
    assert st == adft.ADFT_ERR_ARG, (bad, st, adft.last_error())
    assert not out.value
    assert len(adft.last_error()) > 0


def test_autograd_function_available_without_gpu():
    torch = pytest.importorskip("torch")
    assert issubclass(adft.JKEnergy, torch.autograd.Function)
    assert adft._jk_energy_function() is adft.JKEnergy


def test_header_is_plain_c_and_links_from_c(lib, tmp_path):
    """The boundary is a C ABI: the header compiles as C11 with every warning
    on, and a C program links against the library and calls the entry points
    that need no GPU."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_adft.c"
    src.write_text(
        '#include "adft.h"\n#include <stdio.h>\n#include <string.h>\n'
        "int main(void) {\n"
        "  adft_basis* b = 0;\n"
        "  if (adft_basis_create(0, 0, 0, 0, 1, &b) != ADFT_ERR_ARG || b) return 2;\n"
        "  if (strlen(adft_last_error_message()) == 0) return 3;\n"
        "  printf(\"%s|%s\\n\", adft_version(), adft_status_string(ADFT_ERR_ARG));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "use_adft"
    libdir = os.path.dirname(adft.LIB_PATH)
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-ladft", f"-Wl,-rpath,{libdir}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stderr)
    version, msg = out.stdout.strip().split("|")
    assert version.startswith("adft") and len(msg) > 0


def test_struct_layout_matches_the_binding(tmp_path):
    """The ctypes mirrors of adft_opts, adft_shell and adft_stats have the C
    structs' sizes and field offsets (checked with offsetof in a C program
    compiled against the header)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"adft_opts": adft.adft_opts, "adft_shell": adft.adft_shell, "adft_stats": adft.adft_stats}
    lines = ['#include "adft.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)

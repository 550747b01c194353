"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

No compute call is made here (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"^\s*typedef[^;]*;", "", text, flags=re.M | re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2105_14156_gb300 import build, smash
    build.build()
    return smash.load_library()


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("spgemm_symbolic", "spgemm_numeric", "smash_create", "smash_destroy", "smash_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2105_14156_gb300 import smash
    assert sorted(smash.EXPORTS) == declared_functions()


def test_host_only_calls(lib):
    from paper_2105_14156_gb300 import smash
    p = smash.default_params()
    assert p.max_load == pytest.approx(0.5) and p.hash_kind == 1
    assert lib.smash_status_string(0) == b"SMASH_OK"
    assert lib.smash_status_string(2) == b"SMASH_ERR_SHAPE_MISMATCH"
    # argument checks happen before any device work
    assert lib.smash_create(None, 0, None) == 1
    assert lib.spgemm_symbolic(None, None, None, None, None, None) == 1


STRUCTS = {"smash_csr": "CsrStruct", "smash_params": "Params", "smash_stats": "Stats",
           "smash_kernel_time": "KernelTime", "smash_train_cfg": "TrainCfg",
           "smash_learned_stats": "LearnedStats", "smash_batched_stats": "BatchedStats"}


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    the C compiler gives the header's struct (a host C program, no GPU)."""
    import shutil
    import subprocess
    from paper_2105_14156_gb300 import smash
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "smash.h"', "int main(void) {"]
    expect = []
    for cname, pname in STRUCTS.items():
        cls = getattr(smash, pname)
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
            expect.append(getattr(cls, f).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect

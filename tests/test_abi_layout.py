"""The ctypes mirrors of the structs in include/csc.h match the C layout (offsets and
sizes from a C program compiled against the header with the host compiler), and the
Python wrappers reject wrongly typed tensors before any library call."""
import ctypes
import os
import shutil
import subprocess

import pytest
import torch

from paper_1602_02018_gb300 import _native as nat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {
    "csc_params": nat.csc_params,
    "csc_cluster_info": nat.csc_cluster_info,
    "csc_batch_info": nat.csc_batch_info,
    "csc_cg_info": nat.csc_cg_info,
    "csc_lambda_info": nat.csc_lambda_info,
}
C_FIELD = {"lambda_": "lambda"}  # Python-side renames of C fields


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "csc.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            cf = C_FIELD.get(f, f)
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {cf}));')
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines))
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    return table


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, name):
    cls = STRUCTS[name]
    assert ctypes.sizeof(cls) == c_layout[(name, "size")]
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == c_layout[(name, f)], f"{name}.{f}"


def test_wrappers_reject_wrong_dtypes_before_calling():
    import paper_1602_02018_gb300 as csc

    with pytest.raises(ValueError):
        csc.csc_sample_weighted(torch.zeros(10, dtype=torch.float32), 3)
    with pytest.raises(ValueError):
        csc.csc_coherence_scores(torch.zeros((4, 4), dtype=torch.int32), 4)

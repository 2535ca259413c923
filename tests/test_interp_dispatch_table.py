"""The interpreter's LUT dispatch (interp_device.cuh): an indirect branch
through a table of 256 labels.  Entry i of the table must be the label whose
four lop3.b32 carry the immediate i, for every i, or an instruction would
run another truth table.  Checked on the preprocessed source (no GPU)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1310_6978_b300", "csrc")


def test_jump_table_entries_match_their_immediates(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "t.cu"
    src.write_text('#include "interp_device.cuh"\n')
    out = subprocess.run([nvcc, "-E", "-x", "cu", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}", str(src)],
                         capture_output=True, text=True, check=True).stdout
    text = re.sub(r'"\s*"', "", out)          # join adjacent string literals
    i = text.index(".branchtargets")
    table = re.findall(r"L(0x[0-9A-F]{2})", text[i:text.index(";", i)])
    assert [int(t, 16) for t in table] == list(range(256))
    body = text[text.index(";", i):]
    sep = r"(?:\\n|\\t|\s)*"            # the escapes \n \t of the asm text, as written in the source
    cases = re.findall(r"L(0x[0-9A-F]{2}): ((?:lop3\.b32 %\d, %\d+, %\d+, %\d+, 0x[0-9A-F]{2};" + sep + r"){4})bra\.uni LEND;",
                       body)
    assert len(cases) == 256
    for label, ops in cases:
        imms = re.findall(r"(0x[0-9A-F]{2});", ops)
        assert imms == [label] * 4, (label, imms)
    assert len({label for label, _ in cases}) == 256

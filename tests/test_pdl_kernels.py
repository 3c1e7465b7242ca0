"""Kernels launched with programmatic dependent launch wait for their predecessor.

A kernel launched through ``launch_pdl`` may start while the kernel before it
on the stream is still running; it is correct only if its first statement is
``pdl_begin()`` (griddepcontrol.wait, then the trigger for its own successor).
This reads the CUDA sources and checks every such kernel.
"""

import pathlib
import re

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2503_21176_gb300" / "csrc"


def _sources():
    return {p.name: p.read_text() for p in sorted(CSRC.glob("*.cu"))}


def _launched():
    names = set()
    for text in _sources().values():
        for m in re.finditer(r"launch_pdl\(\s*[^,()]+,\s*(k_\w+)", text):
            names.add(m.group(1))
    return names


def _first_statements(name):
    """First statement of the body of every __global__ definition of ``name``."""
    out = []
    for text in _sources().values():
        for m in re.finditer(r"__global__[^;{}]*?\b" + name + r"\s*\(", text, re.S):
            # the parameter list may contain parentheses: take the brace that
            # follows the matching closing parenthesis of the signature
            depth, k = 1, m.end()
            while depth:
                depth += {"(": 1, ")": -1}.get(text[k], 0)
                k += 1
            body = text.index("{", k)
            stmt = text[body + 1:].lstrip().split(";", 1)[0].strip()
            out.append(stmt)
    return out


def test_some_kernels_use_programmatic_launch():
    names = _launched()
    assert {"k_charges", "k_jacobian", "k_advance", "k_finish"} <= names


def test_every_programmatically_launched_kernel_waits_first():
    for name in sorted(_launched()):
        firsts = _first_statements(name)
        assert firsts, f"{name}: no __global__ definition found"
        for stmt in firsts:
            assert stmt == "pdl_begin()", f"{name} starts with {stmt!r}, not pdl_begin()"

"""Static checks of the CUDA sources (no GPU needed).

A kernel launched with programmatic stream serialization may start while its
predecessor is still running, so it must wait (griddep_wait) before touching
any memory: every kernel passed to launch_pdl has to begin with that call."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1802_09277_gb300", "csrc")


def _sources():
    out = {}
    for name in os.listdir(CSRC):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, name)) as fh:
                out[name] = fh.read()
    return out


def _body_start(src, kernel):
    """Text of the first statements of __global__ kernel `kernel`."""
    m = re.search(r"__global__[^;{]*?\b" + re.escape(kernel) + r"\s*\(", src, re.S)
    if not m:
        return None
    depth, i = 0, m.end() - 1
    while i < len(src):  # skip the parameter list
        if src[i] == "(":
            depth += 1
        elif src[i] == ")":
            depth -= 1
            if depth == 0:
                break
        i += 1
    j = src.index("{", i)
    return src[j + 1:j + 200]


def test_pdl_kernels_wait_first():
    srcs = _sources()
    launched = set()
    for text in srcs.values():
        for m in re.finditer(r"launch_pdl\(\s*([A-Za-z_][A-Za-z0-9_]*)", text):
            launched.add(m.group(1))
    launched -= {"kernel", "void"}  # the helper's own declaration
    assert len(launched) >= 10
    for k in sorted(launched):
        bodies = [b for b in (_body_start(t, k) for t in srcs.values()) if b is not None]
        assert bodies, "definition of %s not found" % k
        for b in bodies:
            first = b.strip().split(";")[0].strip()
            assert first == "griddep_wait()", "%s starts with %r" % (k, first)


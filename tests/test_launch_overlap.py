"""Static check of the launch-overlap invariant (no GPU).

A kernel launched through ``launch_k`` may carry the programmatic-dependent-launch attribute, so
its CTAs can be scheduled while the previous kernel on the stream is still running.  That is only
correct if the kernel waits for its predecessor (``pdl_wait()``, i.e. griddepcontrol.wait) before
its first memory access.  This test reads the CUDA sources and checks that every kernel passed to
``launch_k`` opens its body with ``pdl_wait();``.
"""
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2210_02690_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            out[f] = open(os.path.join(CSRC, f)).read()
    return out


def _launched(src):
    names = set()
    for m in re.finditer(r"launch_k\(\s*([A-Za-z_][A-Za-z0-9_]*)", src):
        names.add(m.group(1))
    return names


def _kernel_bodies(srcs, name):
    pat = re.compile(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s*)?(?:__maxnreg__\([^)]*\)\s*)?"
                     + re.escape(name) + r"\s*\(")
    bodies = []
    for src in srcs.values():
        for m in pat.finditer(src):
            i, depth = m.end() - 1, 0
            while True:
                if src[i] == "(":
                    depth += 1
                elif src[i] == ")":
                    depth -= 1
                    if depth == 0:
                        break
                i += 1
            j = src.index("{", i)
            bodies.append(src[j + 1:j + 200])
    return bodies


def test_every_overlapped_kernel_waits_first():
    srcs = _sources()
    names = set()
    for src in srcs.values():
        names |= _launched(src)
    names.discard("void")  # the declaration of launch_k itself
    assert len(names) >= 15, sorted(names)
    for name in sorted(names):
        bodies = _kernel_bodies(srcs, name)
        assert bodies, f"no __global__ definition found for {name}"
        for body in bodies:
            first = body.strip().split(";")[0].strip()
            assert first == "pdl_wait()", f"{name} does not open with pdl_wait(): {first!r}"


def test_no_raw_launch_of_an_overlapped_kernel():
    """A kernel that opens with pdl_wait() is launched through launch_k only, so that the
    launch counter and the attribute stay in one place."""
    srcs = _sources()
    waiting = set()
    for src in srcs.values():
        for m in re.finditer(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s*)?(?:__maxnreg__\([^)]*\)\s*)?"
                             r"([A-Za-z_][A-Za-z0-9_]*)\s*\(", src):
            waiting.add(m.group(1))
    raw = set()
    for src in srcs.values():
        for m in re.finditer(r"([A-Za-z_][A-Za-z0-9_]*)\s*(?:<[^<>;]*(?:<[^<>;]*>[^<>;]*)*>)?\s*<<<", src):
            raw.add(m.group(1))
    overlapped = {n for n in waiting if any(b.strip().startswith("pdl_wait();") for b in _kernel_bodies(srcs, n))}
    assert not (overlapped & raw), sorted(overlapped & raw)

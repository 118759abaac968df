"""Static check of the programmatic-dependent-launch rule in the CUDA sources:
every kernel launched through launch_pdl() may be scheduled before its
predecessor in the stream has finished, so its body must open with
pdl_enter() (griddepcontrol.wait) before any memory access.  A kernel that
skipped the wait would break the ordering of everything after it."""
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2411_08178_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            out[f] = open(os.path.join(CSRC, f)).read()
    return out


def _kernel_bodies(text):
    """name -> list of body openings (text after the '{' of each __global__)."""
    res = {}
    for m in re.finditer(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s+)?(\w+)\s*\(", text):
        name = m.group(1)
        depth, i = 1, m.end()
        while depth:                       # skip the parameter list
            depth += {"(": 1, ")": -1}.get(text[i], 0)
            i += 1
        j = text.index("{", i)
        res.setdefault(name, []).append(text[j + 1:j + 400])
    return res


def test_every_pdl_launched_kernel_waits_first():
    src = _sources()
    headers = {f: t for f, t in src.items() if f.endswith(".cuh")}
    checked = 0
    for f, t in src.items():
        # a launch refers to a kernel of the same file or of an included header
        # (kernels of the same name in other files live in other anonymous
        # namespaces)
        bodies = dict(_kernel_bodies(t))
        for h, ht in headers.items():
            if f'#include "{h}"' in t or h == f:
                for k, v in _kernel_bodies(ht).items():
                    bodies.setdefault(k, []).extend(v)
        launched = {m.group(1) for m in re.finditer(r"launch_pdl\(\s*(\w+)", t)}
        for m in re.finditer(r"auto\s+(\w+)\s*=\s*(\w+)<", t):   # local alias: auto k = name<...>
            if m.group(1) in launched:
                launched.discard(m.group(1))
                launched.add(m.group(2))
        launched -= {"void", "kernel"}   # the helper's own definition
        for k in sorted(launched):
            assert k in bodies, f"{f}: {k}: no __global__ definition found"
            for body in bodies[k]:
                assert "pdl_enter();" in body, f"{f}: {k} is launched with launch_pdl but does not call pdl_enter()"
                # only declarations may come before the wait
                head = body.split("pdl_enter();")[0]
                for stmt in filter(None, (x.strip() for x in head.split(";"))):
                    assert stmt.startswith(("extern __shared__", "__shared__", "constexpr", "//", "using")), \
                        f"{f}: {k}: '{stmt}' runs before pdl_enter()"
                checked += 1
    assert checked >= 20, checked


def test_launch_helper_sets_the_attribute():
    t = _sources()["internal.cuh"]
    assert "cudaLaunchAttributeProgrammaticStreamSerialization" in t
    assert "griddepcontrol.wait" in t

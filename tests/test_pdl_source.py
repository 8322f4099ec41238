"""Source check of the programmatic-dependent-launch invariant (no GPU needed).

A kernel launched with programmatic stream serialization may be scheduled while
the previous kernel on its stream is still running; it is correct only if its
first statement is pdl_wait() (griddepcontrol.wait), before any access to
global memory.  This test finds every such launch in csrc/ -- launch_dep() calls
and the cluster launches that add the attribute themselves -- resolves the
kernels they can launch, and checks the first statement of each kernel body.
"""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2107_10654_gb300", "csrc")

# kernels launched through a function-pointer variable, by file and variable name
VARIABLE_TARGETS = {
    ("walk.cu", "k"): ["k_walk_dot", "k_walk_dot2", "k_walk_axpy"],
    ("walk.cu", "lanes"): ["k_walk_axpy_lanes", "k_walk_axpy_lanes2"],
    ("gram_tc.cu", "kern"): ["k_tcg_narrow"],
    ("exact.cu", "k"): ["k_ttm_last", "k_ttm_last2w", "k_ttm_mid"],
}
# launches that set cudaLaunchAttributeProgrammaticStreamSerialization by hand
ATTRIBUTE_LAUNCHES = {"sort.cu": ["k_sort_dedupe_cluster"], "kpcg.cu": ["k_kpcg_cluster"]}


def _sources():
    return {os.path.basename(f): open(f).read() for f in glob.glob(os.path.join(CSRC, "*.cu"))}


def _first_statement(src, kernel):
    """First statement of every __global__ definition named `kernel`."""
    out = []
    for m in re.finditer(r"__global__[^;{]*?\b" + re.escape(kernel) + r"\s*\(", src):
        body = src.index("{", m.end())
        # the body opens at the first brace after the parameter list
        stmt = src[body + 1:].lstrip().split("\n", 1)[0].strip()
        out.append(stmt)
    return out


def _launch_targets(srcs):
    targets = []
    for name, src in srcs.items():
        for m in re.finditer(r"launch_dep\(\s*h\s*,\s*([^,]+?)\s*,", src):
            expr = m.group(1)
            names = re.findall(r"\b(k_\w+)", expr)
            if names:
                targets += [(name, n) for n in names]
            else:
                key = (name, expr.strip())
                assert key in VARIABLE_TARGETS, f"unresolved launch_dep target {key}"
                targets += [(name, n) for n in VARIABLE_TARGETS[key]]
    for name, kernels in ATTRIBUTE_LAUNCHES.items():
        assert "cudaLaunchAttributeProgrammaticStreamSerialization" in srcs[name]
        targets += [(name, k) for k in kernels]
    return sorted(set(targets))


def test_every_dependent_launch_waits_first():
    srcs = _sources()
    allsrc = "\n".join(srcs.values())
    targets = _launch_targets(srcs)
    assert len(targets) >= 20
    for fname, kernel in targets:
        firsts = _first_statement(allsrc, kernel)
        assert firsts, f"{kernel} (launched in {fname}) has no __global__ definition"
        for stmt in firsts:
            assert stmt == "pdl_wait();", f"{kernel}: first statement is {stmt!r}"


def test_attribute_only_in_known_places():
    """Every hand-written use of the attribute is one the check above covers."""
    for name, src in _sources().items():
        if "cudaLaunchAttributeProgrammaticStreamSerialization" in src:
            assert name in ATTRIBUTE_LAUNCHES, name
    common = open(os.path.join(CSRC, "common.cuh")).read()
    assert "programmaticStreamSerializationAllowed = 1" in common
    assert "griddepcontrol.wait" in common


def test_no_dependent_launch_behind_an_event_wait():
    """The kernel right after a cross-stream event wait on the main stream is
    launched in full order: the gather, the solve's first CG, the Kronecker
    eigenbasis solve of the exact update."""
    src = _sources()["api.cu"]
    assert src.count("cudaStreamWaitEvent(h->stream, h->ev_join, 0)") == 3
    gather = _sources()["gather.cu"]
    assert "launch_dep(h, k_gather_weights" not in gather
    exact = _sources()["exact.cu"]
    assert "launch_dep(h, k_kron_eig_core" not in exact
    # the first CG solve of a call is launched without the attribute
    assert re.search(r"launch_kpcg\([^;]*!first\)", src, re.S)

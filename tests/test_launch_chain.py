"""Source checks of the step's launch chain (CPU only).

Kernels of the step may be launched with programmatic dependent launch, so
each of them must wait for its predecessor (pdl_enter(): griddepcontrol.wait)
before it touches memory, and before any early return, or a kernel's
completion would no longer imply the completion of the kernels before it.
These tests read the CUDA sources and check that every kernel of the step
starts with pdl_enter() and is launched through launch_chained().
"""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2602_14493_b300", "csrc")

# the kernels of one forward + loss + backward step
STEP_KERNELS = ["k_pad_verts", "k_project", "k_scan_single", "k_scan_reduce", "k_scan_top", "k_scan_down", "k_place_keys",
                "k_tile_sort", "k_long_sort", "k_split_quads", "k_raster_fwd", "k_raster_bwd", "k_sum_partials",
                "k_proj_bwd"]


def _sources():
    out = {}
    for fn in sorted(os.listdir(CSRC)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, fn)) as f:
                out[fn] = f.read()
    return out


def _strip_comments(src):
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.sub(r"//[^\n]*", "", src)


def _kernel_body_start(src, name):
    """First statement of __global__ kernel `name` (None if not defined here)."""
    m = re.search(r"__global__[^;{]*?\b" + name + r"\(", src)
    if not m:
        return None
    depth, i = 0, m.end() - 1
    while True:  # skip the parameter list
        c = src[i]
        depth += c == "("
        depth -= c == ")"
        i += 1
        if depth == 0:
            break
    body = src.index("{", i) + 1
    return src[body:].lstrip().split(";", 1)[0] + ";"


@pytest.mark.parametrize("name", STEP_KERNELS)
def test_step_kernel_waits_for_its_predecessor_first(name):
    found = [(fn, _kernel_body_start(_strip_comments(src), name)) for fn, src in _sources().items()]
    found = [(fn, st) for fn, st in found if st is not None]
    assert len(found) == 1, f"{name} defined {len(found)} times"
    fn, first = found[0]
    assert first == "pdl_enter();", f"{name} in {fn} starts with {first!r}"


def test_step_kernels_not_launched_with_triple_chevrons():
    for fn, src in _sources().items():
        code = _strip_comments(src)
        for name in STEP_KERNELS:
            assert not re.search(r"\b" + name + r"\s*(<[^;]*?>)?\s*<<<", code), f"{name} launched with <<< in {fn}"


def test_chained_launch_sites_name_step_kernels():
    srcs = {fn: _strip_comments(s) for fn, s in _sources().items()}
    sites = [(fn, m.group(1), m.group(2)) for fn, s in srcs.items()
             for m in re.finditer(r"launch_chained\((\w+),\s*(true|false)", s)]
    assert sites, "no chained launches found"
    # 'kern' is a local pointer to one instantiation of a step kernel template
    for fn, kern, _ in sites:
        assert kern in STEP_KERNELS or kern == "kern", (fn, kern)
    # kernels whose CTAs take tiles heaviest first are launched unchained
    for fn, kern, chained in sites:
        if kern == "k_tile_sort" or (kern == "kern" and fn == "gmr_raster.cu"):
            assert chained == "false", (fn, kern)

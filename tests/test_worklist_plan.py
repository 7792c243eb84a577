"""Host side of work-list batches (tucker_batch_describe; no GPU): the phases and
grouped launches a batch becomes, the planner's own dependency and extent
checks on random batches, the workspace it adds, and the batches it refuses."""
import re

import numpy as np
import pytest
import torch

from paper_2303_11612_gb300 import _binding as B


def parse(text):
    steps, groups, lanes = [], [], []
    for line in text.strip().splitlines():
        m = re.match(r"step (\d+) lane (\d+): items=(\d+) init=(\d+) gaussian=(\d+) power=(\d+) sum=(\d+) "
                     r"product=(\d+) smem=(\d+) heavy=(\d+)", line)
        if m:
            v = [int(x) for x in m.groups()]
            steps.append(tuple([v[0]] + v[2:9]))
            lanes.append(v[1])
            groups.append("step")
            continue
        m = re.match(r"(cholqr|extract) lane (\d+): jobs=(\d+)", line)
        if m:
            groups.append((m.group(1), int(m.group(3))))
            lanes.append(int(m.group(2)))
            continue
        m = re.match(r"lanes=(\d+) tasks=(\d+) items=(\d+) area=(\d+)", line)
        assert m, line
        nl = int(m.group(1))
        total = tuple(int(x) for x in m.groups()[1:])
    assert sorted(set(lanes)) == list(range(nl)) and lanes == sorted(lanes)   # lane by lane
    return steps, groups, total


def expected_steps(specs):
    """Phases per lane: per mode one (truncation, status reset, Omega) and two per power
    step (partials, sums) for the longest power iteration among the lane's requests on
    that mode; then one per position of the core chains that has a product."""
    nl = max(1, min(8, len(specs) // 4))
    total = 0
    for lane in range(nl):
        mem = specs[lane::nl]
        maxN = max(len(s["dims"]) for s in mem)
        total += sum(1 + 2 * max(s["q"] for s in mem if len(s["dims"]) > m) for m in range(maxN))
        total += sum(1 for m in range(maxN)
                     if any((s["which"] == "T" and m < len(s["dims"])) or (s["which"] == "ST" and m == len(s["dims"]) - 1)
                            for s in mem))
    return total


def test_st_hosvd_steps():
    # 64 x 48 x 40, ranks (8, 6, 5), q = 1: per mode a phase with the status reset (first
    # mode) or the truncation by U_{n-1} (later modes) and Omega_n, a phase of power-step
    # partials, a phase of their sums, then the grouped extraction; a last phase forms the core
    steps, groups, (tasks, items, area) = parse(B.batch_describe([dict(which="ST", dims=(64, 48, 40),
                                                                       ranks=(8, 6, 5), P=4, q=1)]))
    mode = ["step", "step", "step", ("extract", 1)]
    assert groups == mode * 3 + ["step"]
    assert [s[2:7] for s in steps] == [(1, 1, 0, 0, 0), (0, 0, 1, 0, 0), (0, 0, 0, 1, 0)] + \
        [(0, 1, 0, 0, 1), (0, 0, 1, 0, 0), (0, 0, 0, 1, 0)] * 2 + [(0, 0, 0, 0, 1)]
    # the core: the product by U_3 of the 8 x 6 x 40 tensor (48 fibers, one block of 128)
    assert steps[-1][1] == 1
    # the product by U_1: 48 * 40 fibers in blocks of 128, 8 outputs in one block; and Omega_2
    assert steps[3][1] == 15 + 1
    assert tasks == sum(sum(s[2:7]) for s in steps) and items == sum(s[1] for s in steps)
    assert area % 256 == 0 and area > 0


@pytest.mark.parametrize("q", [1, 2, 3])
def test_t_hosvd_steps(q):
    N = 4
    steps, groups, _ = parse(B.batch_describe([dict(which="T", dims=(20, 18, 16, 14), ranks=(4, 3, 3, 2), P=2,
                                                    q=q)]))
    # per mode: q steps with a CholeskyQR between consecutive ones, then the extraction;
    # then one step with the whole core chain
    want = []
    for _ in range(N):
        want.append("step")                                  # (status reset,) Omega_n
        for k in range(q):
            if k:
                want.append(("cholqr", 1))
            want += ["step", "step"]                         # partials, sums
        want.append(("extract", 1))
    want += ["step"] * N                                     # the core chain, a phase per product
    assert groups == want
    assert len(steps) == N * (1 + 2 * q) + N
    assert all(s[2:7] == (0, 0, 0, 0, 1) for s in steps[-N:])
    assert sum(s[3] for s in steps) == N                     # one Gaussian per mode
    assert sum(s[4] for s in steps) == N * q                 # one power task per power step


def test_batches_group_every_request():
    specs = [dict(which="ST", dims=(64, 48, 40), ranks=(8, 6, 5), P=4, q=1),
             dict(which="T", dims=(30, 28, 26, 24), ranks=(4, 4, 3, 2), P=3, q=2),
             dict(which="ST", dims=(256, 17, 33), ranks=(32, 5, 7), P=8, q=2)]
    steps, groups, _ = parse(B.batch_describe(specs))
    # the longest requests set the schedule: 4 modes of (1 + 2 x 2) phases, 4 core phases
    assert len(steps) == expected_steps(specs) == 24
    assert groups.count(("extract", 3)) == 3 and ("extract", 1) in groups
    # CholeskyQR between power steps only for the q = 2 requests still on their modes
    assert ("cholqr", 2) in groups and ("cholqr", 1) in groups
    assert sum(s[2] for s in steps) == 3                     # one status reset per request


def test_random_batches_pass_the_dependency_check():
    rng = np.random.default_rng(0)
    for trial in range(40):
        specs = []
        for k in range(int(rng.integers(1, 24))):
            N = int(rng.integers(1, 6))
            dims = [int(x) for x in rng.integers(1, 257 if N <= 3 else 33, size=N)]
            ranks = [int(min(d, x)) for d, x in zip(dims, rng.integers(1, 33, size=N))]
            specs.append(dict(which="ST" if rng.random() < 0.5 else "T", dims=dims, ranks=ranks,
                              P=int(rng.integers(0, 10)), q=int(rng.integers(1, 4)), seed=k))
        dtype = torch.float32 if trial % 2 == 0 else torch.float64
        steps, groups, (tasks, items, area) = parse(B.batch_describe(specs, dtype=dtype))
        assert len(steps) == expected_steps(specs)
        assert items == sum(s[1] for s in steps) and tasks == sum(sum(s[2:7]) for s in steps)
        assert all(s[7] <= 227 * 1024 for s in steps)


def test_requests_are_dealt_to_lanes():
    specs = [dict(which="ST", dims=(40, 30, 20), ranks=(4, 3, 2), P=2, q=1, seed=k) for k in range(13)]
    out = B.batch_describe(specs)
    assert "lanes=3 " in out
    steps, groups, _ = parse(out)
    # each lane: 3 modes (three phases and an extraction each) and the core phase
    assert len(steps) == 3 * 10 == expected_steps(specs)
    assert [g for g in groups if g != "step"] == [("extract", 5)] * 3 + [("extract", 4)] * 6


def test_workspace_adds_the_descriptor_area():
    import ctypes as C
    specs = [dict(which="ST", dims=(64, 48, 40), ranks=(8, 6, 5), P=4, q=1),
             dict(which="T", dims=(32, 30, 28), ranks=(4, 4, 3), P=2, q=1)]
    arr = (B.Request * 2)()
    keep = []
    for k, r in enumerate(specs):
        d64, r32 = B._i64(r["dims"]), B._i32(r["ranks"])
        Up = (C.c_void_p * 3)(256, 256, 256)
        arr[k] = B.Request(C.sizeof(B.Request), 1 if r["which"] == "ST" else 0, 0, 256, d64, 3, r32, r["P"], r["q"],
                           0, 1, 0, Up, 256)
        keep.append((d64, r32, Up))
    sizes = []
    for flags in (0, B.FLAG_WORKLIST):
        o = B.make_opts(flags=flags)
        n = C.c_size_t(0)
        assert B.lib().tucker_batch_workspace_size(2, C.cast(arr, C.c_void_p), C.byref(o), C.byref(n)) == 0
        sizes.append(n.value)
    area = parse(B.batch_describe(specs))[2][2]
    assert sizes[1] == sizes[0] + area


@pytest.mark.parametrize("spec,kw", [
    (dict(which="ST", dims=(300, 20, 20), ranks=(4, 4, 4)), {}),            # extent > 256
    (dict(which="T", dims=(64, 64, 64), ranks=(40, 4, 4)), {}),             # rank > 32
    (dict(which="ST", dims=(64, 64, 64), ranks=(4, 4, 4), c=100), {}),      # sampling (Algorithm 5)
    (dict(which="ST", dims=(64, 64, 64), ranks=(4, 4, 4)), dict(prec="bf16")),
    (dict(which="ST", dims=(64, 64, 64), ranks=(4, 4, 4)), dict(prec="tf32")),
    (dict(which="ST", dims=(64, 64, 64), ranks=(4, 4, 4)), dict(form="range")),
], ids=["extent", "rank", "amm", "bf16", "tf32", "range"])
def test_unsupported_batches_are_refused(spec, kw):
    with pytest.raises(B.TuckerError) as e:
        B.batch_describe([spec], **kw)
    assert e.value.status == 6                                              # TUCKER_ERR_UNSUPPORTED


def test_mixed_element_types_are_refused():
    import ctypes as C
    arr = (B.Request * 2)()
    keep = []
    for k in range(2):
        d64, r32 = B._i64((20, 20, 20)), B._i32((3, 3, 3))
        Up = (C.c_void_p * 3)(256, 256, 256)
        arr[k] = B.Request(C.sizeof(B.Request), 1, k, 256, d64, 3, r32, 2, 1, 0, 1, 0, Up, 256)
        keep.append((d64, r32, Up))
    o = B.make_opts(flags=B.FLAG_WORKLIST)
    buf = C.create_string_buffer(4096)
    assert B.lib().tucker_batch_describe(2, C.cast(arr, C.c_void_p), C.byref(o), buf, len(buf)) == 6


def test_the_work_list_is_not_run():
    """tucker_batch_run refuses TUCKER_FLAG_WORKLIST before any launch (the path is
    planned but kept off the device), and the server refuses ticks."""
    import ctypes as C
    arr = (B.Request * 1)()
    d64, r32 = B._i64((20, 20, 20)), B._i32((3, 3, 3))
    Up = (C.c_void_p * 3)(256, 256, 256)
    arr[0] = B.Request(C.sizeof(B.Request), 1, 0, 256, d64, 3, r32, 2, 1, 0, 1, 0, Up, 256)
    o = B.make_opts(flags=B.FLAG_WORKLIST)
    o.workspace = 256
    o.workspace_bytes = 1 << 30
    assert B.lib().tucker_batch_run(1, C.cast(arr, C.c_void_p), C.byref(o)) == 6
    so = B.ServerOpts(C.sizeof(B.ServerOpts), 8, 1 << 30, 0, 0, 8, 1 << 20)
    h = C.c_void_p()
    assert B.lib().tucker_server_create(C.byref(so), C.byref(h)) == 6 and not h.value

"""The C-ABI library loads and exports every entry point include/tucker.h
declares; host-side argument checks reject bad input before any launch.
Runs without a GPU (no compute calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:tucker_status|const char\*|int64_t)\s+(tucker_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2303_11612_gb300 import _binding
    return _binding.lib()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("tucker_rthosvd", "tucker_rsthosvd", "tucker_workspace_size", "tucker_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2303_11612_gb300 import _binding
    assert set(declared()) <= set(_binding.exported_symbols())


def test_status_strings(lib):
    for s in range(8):
        assert lib.tucker_status_string(s)


def _ws(lib, dims, ranks, P=10, q=1, c=0, which=1):
    from paper_2303_11612_gb300 import _binding as B
    n = C.c_size_t(0)
    st = lib.tucker_workspace_size(which, 0, B._i64(dims), len(dims), B._i32(ranks), P, q, c, None, C.byref(n))
    return st, n.value


def test_workspace_size_and_argument_checks(lib):
    st, n = _ws(lib, (400, 400, 400), (20, 20, 20))
    assert st == 0 and n > 0
    st2, n2 = _ws(lib, (400, 400, 400), (20, 20, 20), c=4000)
    assert st2 == 0 and n2 > n                   # AMM buffers
    assert _ws(lib, (400, 400, 400), (401, 20, 20))[0] == 1       # R > I
    assert _ws(lib, (400, 400, 400), (0, 20, 20))[0] == 1         # R < 1
    assert _ws(lib, (400, 400, 400), (20, 20, 20), q=0)[0] == 1   # q < 1
    assert _ws(lib, (400, 400, 400), (20, 20, 20), P=-1)[0] == 1  # P < 0
    assert _ws(lib, (4096, 8, 8), (4, 4, 4))[0] == 6             # I_n beyond the built limit
    assert _ws(lib, (), ())[0] == 1


def test_drivers_reject_bad_arguments_without_touching_memory(lib):
    from paper_2303_11612_gb300 import _binding as B
    U = (C.c_void_p * 3)(1, 1, 1)
    # rank larger than the dimension: rejected before any CUDA call
    st = lib.tucker_rsthosvd(C.c_void_p(1), 0, B._i64((10, 10, 10)), 3, B._i32((11, 2, 2)), 5, 1, 0, 1,
                             C.c_uint64(0), U, C.c_void_p(1), None)
    assert st == 1
    st = lib.tucker_rthosvd(None, 0, B._i64((10, 10, 10)), 3, B._i32((2, 2, 2)), 5, 1, 0, 1,
                            C.c_uint64(0), U, C.c_void_p(1), None)
    assert st == 1
    o = B.make_opts()
    o.struct_size = 4                                  # too small
    st = lib.tucker_rsthosvd(C.c_void_p(1), 0, B._i64((10, 10, 10)), 3, B._i32((2, 2, 2)), 5, 1, 0, 1,
                             C.c_uint64(0), U, C.c_void_p(1), C.byref(o))
    assert st == 1


def _request(dims, ranks, which=1, N=None, P=10, q=1, c=0):
    from paper_2303_11612_gb300 import _binding as B
    r = B.Request()
    r.struct_size = C.sizeof(B.Request)
    r.which, r.dt, r.A, r.G = which, 0, 1, 1
    d, rk = B._i64(dims or (1,)), B._i32(ranks or (1,))
    U = (C.c_void_p * max(1, len(dims)))(*([1] * max(1, len(dims))))
    r.dims = C.cast(d, C.POINTER(C.c_int64))
    r.ranks = C.cast(rk, C.POINTER(C.c_int32))
    r.U = C.cast(U, C.POINTER(C.c_void_p))
    r.N = len(dims) if N is None else N
    r.P, r.q, r.c, r.prob, r.seed = P, q, c, 1, 0
    return r, (d, rk, U)


def test_batch_sizes_and_argument_checks(lib):
    """tucker_batch_workspace_size sums each request's workspace rounded up to
    256 bytes and rejects malformed requests; tucker_batch_run refuses missing
    options or workspace before any CUDA call."""
    from paper_2303_11612_gb300 import _binding as B
    a, ka = _request((400, 400, 400), (20, 20, 20))
    b, kb = _request((64, 48, 40, 36), (8, 6, 5, 4), which=0, c=300)
    arr = (B.Request * 2)(a, b)
    n = C.c_size_t(0)
    assert lib.tucker_batch_workspace_size(2, arr, None, C.byref(n)) == 0
    wa = _ws(lib, (400, 400, 400), (20, 20, 20))[1]
    wb = _ws(lib, (64, 48, 40, 36), (8, 6, 5, 4), which=0, c=300)[1]
    up = lambda x: (x + 255) // 256 * 256
    assert n.value == up(wa) + up(wb)
    assert lib.tucker_batch_workspace_size(0, arr, None, C.byref(n)) == 1
    assert lib.tucker_batch_workspace_size(2, None, None, C.byref(n)) == 1
    assert lib.tucker_batch_workspace_size(2, arr, None, None) == 1
    for bad in (dict(which=2), dict(N=0), dict(q=0), dict(P=-1)):
        r, keep = _request((40, 36, 32), (4, 4, 4), **bad)
        one = (B.Request * 1)(r)
        assert lib.tucker_batch_workspace_size(1, one, None, C.byref(n)) == 1, bad
    r, keep = _request((40, 36, 32), (41, 4, 4))                     # R > I
    assert lib.tucker_batch_workspace_size(1, (B.Request * 1)(r), None, C.byref(n)) == 1
    assert lib.tucker_batch_run(2, arr, None) == 1                     # options (and workspace) required
    o = B.make_opts()
    assert lib.tucker_batch_run(2, arr, C.byref(o)) == 1               # no workspace
    o.prec = 9
    assert lib.tucker_batch_workspace_size(2, arr, C.byref(o), C.byref(n)) == 1


def test_options_and_server_argument_checks(lib):
    """Out-of-range options and server settings are rejected on the host."""
    from paper_2303_11612_gb300 import _binding as B
    for field, value in (("prec", 4), ("prec", -1), ("form", 3), ("alpha", 1.5), ("alpha", -0.1)):
        o = B.make_opts()
        setattr(o, field, value)
        st = lib.tucker_workspace_size(1, 0, B._i64((40, 36, 32)), 3, B._i32((4, 4, 4)), 5, 1, 0, C.byref(o),
                                       C.byref(C.c_size_t()))
        assert st == 1, (field, value)
    h = C.c_void_p()
    assert lib.tucker_server_create(None, C.byref(h)) == 1
    for field, value in (("max_inflight", 0), ("max_inflight", 257), ("budget_bytes", 0), ("form", 3),
                         ("prec", 4)):
        so = B.ServerOpts(C.sizeof(B.ServerOpts), 8, 1 << 30, 0, 0)
        setattr(so, field, value)
        assert lib.tucker_server_create(C.byref(so), C.byref(h)) == 1, (field, value)
    # ticks: invalid settings are refused as such, valid ones as unsupported (the work-list
    # path they would run is not run)
    for tick_max, tick_elems, prec, want in ((300, 1000, 0, 1), (-1, 1000, 0, 1), (4, 0, 0, 1), (4, 1000, 2, 6),
                                              (4, 1000, 0, 6)):
        so = B.ServerOpts(C.sizeof(B.ServerOpts), 8, 1 << 30, 0, prec, tick_max, tick_elems)
        assert lib.tucker_server_create(C.byref(so), C.byref(h)) == want, (tick_max, tick_elems, prec)


def test_noalloc_power_step_checks_options_like_the_power_step(lib):
    """The allocation-free power step answers option errors before any CUDA
    call, with the statuses of tucker_power_step, and refuses the tensor-core
    forms (it serves only the exact FMA arithmetic)."""
    from paper_2303_11612_gb300 import _binding as B
    dims = B._i64((64, 8, 8))
    fake = 0x1000                    # never dereferenced: every case returns before any launch
    bad_form = B.make_opts()
    bad_form.form = 7
    bad_prec = B.make_opts()
    bad_prec.prec = 9
    bad_alpha = B.make_opts(alpha=2.0)
    short = B.make_opts()
    short.struct_size = 8
    for o in (bad_form, bad_prec, bad_alpha, short):
        assert lib.tucker_power_step_noalloc(fake, 0, dims, 3, 0, fake, 8, fake, C.byref(o)) == 1
        assert lib.tucker_power_step(fake, 0, dims, 3, 0, fake, 8, fake, C.byref(o)) == 1
    for prec in ("tf32", "bf16", "bf16x1"):
        o = B.make_opts(prec=prec)
        assert lib.tucker_power_step_noalloc(fake, 0, dims, 3, 0, fake, 8, fake, C.byref(o)) == 6


def test_measurement_entry_points_without_gpu(lib):
    """Launch counter, per-class profile counters (zero before any launch, one
    slot per kernel class the binding names) and the last-CUDA-error string
    answer without a GPU; an unknown class is an argument error."""
    from paper_2303_11612_gb300 import _binding as B
    assert lib.tucker_launch_count() >= 0
    assert lib.tucker_profile_enable(1) == 0
    n, ms, by, fl = C.c_int64(-1), C.c_double(-1), C.c_double(-1), C.c_double(-1)
    classes = sorted(B.KERNEL_CLASSES.values())
    assert classes == list(range(len(classes)))
    for k in classes:
        assert lib.tucker_profile_read(k, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)) == 0
        assert (n.value, ms.value, by.value, fl.value) == (0, 0.0, 0.0, 0.0)
    assert lib.tucker_profile_read(len(classes), None, None, None, None) == 1
    assert lib.tucker_profile_read(-1, None, None, None, None) == 1
    assert lib.tucker_profile_enable(0) == 0
    assert lib.tucker_last_cuda_error() is not None


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "tucker.h"

int main(void) {
    int64_t dims[3] = {400, 400, 400};
    int32_t ranks[3] = {20, 20, 20}, bad[3] = {401, 20, 20};
    size_t bytes = 0;
    if (tucker_workspace_size(1, TUCKER_F32, dims, 3, ranks, 10, 1, 0, NULL, &bytes) != TUCKER_OK || bytes == 0)
        return 1;
    if (tucker_workspace_size(1, TUCKER_F32, dims, 3, bad, 10, 1, 0, NULL, &bytes) != TUCKER_ERR_INVALID_ARG)
        return 2;
    void* U[3] = {NULL, NULL, NULL};
    if (tucker_rsthosvd(NULL, TUCKER_F32, dims, 3, ranks, 10, 1, 0, TUCKER_PROB_UNIFORM, 0, U, NULL, NULL) !=
        TUCKER_ERR_INVALID_ARG)
        return 3;
    tucker_request req;
    memset(&req, 0, sizeof(req));
    req.struct_size = sizeof(req);
    req.which = 1;
    req.dt = TUCKER_F32;
    req.A = dims;                       /* never read: sizing only */
    req.dims = dims;
    req.N = 3;
    req.ranks = ranks;
    req.P = 10;
    req.q = 1;
    req.prob = TUCKER_PROB_UNIFORM;
    req.U = U;
    req.G = dims;
    size_t batch = 0;
    if (tucker_batch_workspace_size(1, &req, NULL, &batch) != TUCKER_OK || batch < bytes) return 4;
    tucker_server_opts so;
    memset(&so, 0, sizeof(so));
    so.struct_size = sizeof(so);
    tucker_server* srv = NULL;
    if (tucker_server_create(&so, &srv) != TUCKER_ERR_INVALID_ARG || srv) return 5;   /* max_inflight 0 */
    printf("%s %zu %zu %lld\n", tucker_status_string(TUCKER_OK), bytes, batch, (long long)tucker_launch_count());
    return 0;
}
"""


def test_plain_c_caller(tmp_path):
    """include/tucker.h is plain C (C99, -pedantic, no warnings) and a C program
    links against the library and gets the documented answers from the host-side
    entry points."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2303_11612_gb300 import _binding as B
    B.lib()
    libdir = os.path.join(ROOT, "paper_2303_11612_gb300", "_lib")
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    cc = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                         str(src), "-L", libdir, "-ltucker", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    assert run.stdout.split()[0] == "ok"


def _modes(text):
    """{mode: {key: value}} from tucker_plan_describe's lines."""
    out = {}
    for line in text.strip().splitlines():
        head, rest = line.split(":", 1)
        out[int(head.split()[1])] = dict(kv.split("=") for kv in rest.split())
    return out


def test_plan_describe_pins_the_dispatch_rules():
    """The arithmetic of each mode, decided on the host: single-pass BF16
    sketches only the input tensor (every T-HOSVD mode, ST-HOSVD's first),
    ST-HOSVD's later (truncated) modes and the TF32 form's strided modes take
    split BF16, the mode product runs split BF16 on contiguous fibers in every
    tensor-core form and FP32 FMA elsewhere, shapes beyond the fused tiles take
    the two-pass tensor-core kernels on contiguous fibers, and FP64 data stays
    FP64."""
    import torch
    from paper_2303_11612_gb300 import _binding as B
    dims, ranks = (400, 400, 400), (20, 20, 20)
    st = _modes(B.plan_describe("ST", dims, ranks, prec="bf16x1"))
    assert [st[n]["power"] for n in range(3)] == ["bf16x1", "split-bf16", "split-bf16"]
    assert [st[n]["ttm"] for n in range(3)] == ["split-bf16", "fp32", "fp32"]
    assert [int(st[n]["J"]) for n in range(3)] == [160000, 20 * 400, 20 * 20]     # ST truncates
    t = _modes(B.plan_describe("T", dims, ranks, prec="bf16x1"))
    assert [t[n]["power"] for n in range(3)] == ["bf16x1"] * 3
    assert [t[n]["sketch"] for n in range(3)] == ["contiguous", "strided", "strided"]
    assert [int(t[n]["J"]) for n in range(3)] == [160000] * 3
    tf = _modes(B.plan_describe("T", dims, ranks, prec="tf32"))
    assert [tf[n]["power"] for n in range(3)] == ["tf32", "split-bf16", "split-bf16"]
    fp = _modes(B.plan_describe("ST", dims, ranks, prec="fp32"))
    assert all(fp[n]["power"] == "fp32" and fp[n]["ttm"] == "fp32" for n in range(3))
    amm = _modes(B.plan_describe("ST", dims, ranks, c=4000, prec="bf16x1"))
    assert [int(amm[n]["T"]) for n in range(3)] == [4000, 4000, 400]               # T_n = min(c, J_n)
    assert all(amm[n]["sketch"] == "contiguous" for n in range(3))                 # the I x T gather
    f64 = _modes(B.plan_describe("ST", (100, 100, 100), (10, 10, 10), P=5, dtype=torch.float64))
    assert all(f64[n]["power"] == "fp64" and f64[n]["ttm"] == "fp64" for n in range(3))
    assert all(int(f64[n]["L"]) == 15 for n in range(3))
    rng = _modes(B.plan_describe("ST", dims, ranks, form="range", prec="bf16x1"))
    # the range form's first pass Y = A Omega: tensor cores on contiguous fibers
    assert [rng[n]["range-sketch"] for n in range(3)] == ["wide-bf16x1", "fp32", "fp32"]
    # beyond the fused tiles (I_n = 1024, L = 80, R = 64): two tensor-core passes on
    # contiguous fibers and the gathered samples, single-pass BF16 on the input tensor only
    big, bigr = (1024, 1024, 512), (64, 64, 32)
    # (strided fibers too where the stride is a multiple of 32: modes 2 and 3 here)
    w1 = _modes(B.plan_describe("ST", big, bigr, P=16, prec="bf16x1"))
    assert [w1[n]["power"] for n in range(3)] == ["wide-bf16x1", "wide-split-bf16", "split-bf16"]
    assert [w1[n]["ttm"] for n in range(3)] == ["wide-split-bf16"] * 3
    assert [int(w1[n]["L"]) for n in range(3)] == [80, 80, 48]
    for prec in ("bf16", "tf32"):
        w2 = _modes(B.plan_describe("ST", big, bigr, P=16, prec=prec))
        assert [w2[n]["power"] for n in range(3)] == ["wide-split-bf16", "wide-split-bf16", "split-bf16"]
    wt = _modes(B.plan_describe("T", big, bigr, P=16, prec="bf16x1"))
    assert [wt[n]["power"] for n in range(3)] == ["wide-bf16x1"] * 3          # every mode sketches the input
    # AMM in the paper form: the gathered sample is sketched in orthonormalised half
    # steps, FP32-class: split bf16 on the tensor cores for samples beyond the fused
    # tiles in the tensor-core forms, FMA otherwise
    wa = _modes(B.plan_describe("ST", big, bigr, P=16, c=20000, prec="bf16x1"))
    assert [wa[n]["power"] for n in range(3)] == ["wide-split-bf16", "wide-split-bf16", "fp32"]
    wf = _modes(B.plan_describe("ST", big, bigr, P=16, c=20000, prec="fp32"))
    assert [wf[n]["power"] for n in range(3)] == ["fp32"] * 3
    assert [wa[n]["amm"] for n in range(3)] == ["half-steps"] * 3
    # Strategy B: with q >= 2 in a tensor-core form, I_n <= 128 and a layout the tensor-core
    # kernels take, G = A_(n) A_(n)^T in one pass replaces the q passes of Strategy A
    qb = _modes(B.plan_describe("ST", (96, 96, 96, 96), (16,) * 4, P=8, q=2, prec="bf16x1"))
    # (ST-HOSVD's mode 2 has the stride R_1 = 16, not a multiple of 32: Strategy A there)
    assert [qb[n]["power"] for n in range(4)] == ["gram-split-bf16", "split-bf16", "gram-split-bf16",
                                                  "gram-split-bf16"]
    qt = _modes(B.plan_describe("T", (96, 96, 96, 96), (16,) * 4, P=8, q=2, prec="tf32"))
    assert [qt[n]["power"] for n in range(4)] == ["gram-split-bf16"] * 4
    q1 = _modes(B.plan_describe("T", (96, 96, 96, 96), (16,) * 4, P=8, q=1, prec="tf32"))
    assert "gram-split-bf16" not in [q1[n]["power"] for n in range(4)]          # q = 1: one pass either way
    qf = _modes(B.plan_describe("T", (96, 96, 96, 96), (16,) * 4, P=8, q=2, prec="fp32"))
    assert [qf[n]["power"] for n in range(4)] == ["fp32"] * 4
    assert [int(wa[n]["T"]) for n in range(3)] == [20000, 20000, 64 * 64]
    # no half steps where the sample has fewer fibers than the sketch has columns
    few = _modes(B.plan_describe("ST", (40, 36, 32), (8, 6, 7), P=5, c=10, prec="bf16x1"))
    assert all("amm" not in few[n] for n in range(3))
    wf = _modes(B.plan_describe("ST", big, bigr, P=16, prec="fp32"))
    assert all(wf[n]["power"] == "fp32" and wf[n]["ttm"] == "fp32" for n in range(3))
    lib = B.lib()
    small = C.create_string_buffer(16)
    assert lib.tucker_plan_describe(1, 0, B._i64(dims), 3, B._i32(ranks), 10, 1, 0, None, small, 16) == 1
    assert lib.tucker_plan_describe(1, 0, B._i64(dims), 3, B._i32((401, 20, 20)), 10, 1, 0, None,
                                    C.create_string_buffer(1024), 1024) == 1


def test_planner_sketch_width_follows_the_oracles_reading():
    """L_n = min(R_n + P, I_n), the reading the oracle takes, in the C planner
    too (for ST-HOSVD on the truncated extents of the earlier modes)."""
    from paper_2303_11612_gb300 import _binding as B
    from oracle import tucker as ot
    dims, ranks, P = (16, 40, 40), (12, 5, 30), 10
    got = _modes(B.plan_describe("ST", dims, ranks, P=P))
    assert [int(got[n]["L"]) for n in range(3)] == [min(r + P, d) for r, d in zip(ranks, dims)] == [16, 15, 40]
    import numpy as np
    A = np.random.default_rng(0).standard_normal(dims)
    info = {}
    ot.rsthosvd(A, ranks, P=P, q=1, info=info)
    assert [info["L"][n] for n in range(3)] == [16, 15, 40]


def test_planner_sample_counts_follow_the_oracle():
    """T_n = min(c, J_n) for c > 0 and ceil(alpha J_n) for c = 0, alpha > 0 (the
    parameter rule of Section 3.3), in the C planner as in the oracle, on the
    tensor each mode works on."""
    from paper_2303_11612_gb300 import _binding as B
    from oracle import tucker as ot
    dims, ranks = (30, 40, 50), (5, 6, 7)
    for which in ("T", "ST"):
        for c, alpha in ((1000, 0.0), (10, 0.0), (0, 0.05), (0, 0.3333), (0, 0.0)):
            got = _modes(B.plan_describe(which, dims, ranks, P=3, c=c, alpha=alpha))
            cur = list(dims)
            for n in range(3):
                J = 1
                for m in range(3):
                    if m != n:
                        J *= cur[m]
                assert int(got[n]["J"]) == J
                assert int(got[n]["T"]) == ot.sample_count(c, alpha, J), (which, c, alpha, n)
                if which == "ST":
                    cur[n] = ranks[n]

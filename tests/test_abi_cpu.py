"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every declared symbol, and the host plan computes the paper's sizes."""
import ctypes as C
import os
import re

import pytest

from paper_2111_10448_gb300 import _native as N

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ttsketch.h")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tt_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = N.lib()
    decl = declared_symbols()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(N.EXPORTED) == decl


def plan(dims, **kw):
    q = N.make_problem(dims, **kw)
    h = C.c_void_p()
    st = N.lib().tt_sketch_plan(C.byref(q), C.byref(h))
    return st, h


def sizes(h):
    ws, ce, re_ = C.c_size_t(), C.c_int64(), C.c_int()
    N.check(N.lib().tt_plan_sizes(h, C.byref(ws), C.byref(ce), C.byref(re_)), "sizes")
    return ws.value, ce.value, re_.value


def layout(h, item=0):
    off = (C.c_int64 * (N.TT_MAXD + 1))()
    rp = (C.c_int * (N.TT_MAXD + 1))()
    N.check(N.lib().tt_plan_core_layout(h, item, off, rp), "layout")
    return list(off), list(rp)


def sketch_list(h, item=0):
    out = []
    i = 0
    while True:
        ty, k, w, rows, off = C.c_int(), C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
        if N.lib().tt_plan_sketch_info(h, item, i, C.byref(ty), C.byref(k), C.byref(rows), C.byref(w),
                                       C.byref(off)) != N.TT_OK:
            return out
        out.append((ty.value, k.value, rows.value, w.value, off.value))
        i += 1


def test_table1_core_storage_through_plan(golden):
    """Table 1 TT sizes, computed by the plan's core layout (fixed ranks)."""
    for d, n, ranks, gb, mb in golden("table1_sizes.txt"):
        d, n = int(d), int(n)
        r = [int(v) for v in ranks.split(",")]
        st, h = plan([n] * d, ranks=r, p=2)
        assert st == N.TT_OK
        _, ce, re_ = sizes(h)
        assert f"{ce * 8 / 2 ** 20:.3g}" == f"{float(mb):.3g}"
        assert re_ == d + 1
        N.lib().tt_plan_destroy(h)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 9])
def test_split_and_sketch_list(d):
    """d* = ceil(d/2); column sketches k < d* (+ the middle one in one-pass),
    row sketches k = d*..d-1 (the dimensionally consistent reading of the
    middle-core formula); widths l = r + p."""
    dims = [3 + (k % 3) for k in range(d)]
    r = [1] + [2] * (d - 1) + [1]
    ds = (d + 1) // 2
    Nk = [1]
    for n in dims:
        Nk.append(Nk[-1] * n)
    for passes in (1, 2):
        st, h = plan(dims, ranks=r, p=3, passes=passes)
        assert st == N.TT_OK
        sk = sketch_list(h)
        want = [(0, k, Nk[k]) for k in range(1, ds)]
        if passes == 1:
            want.append((0, ds, Nk[ds]))
        want += [(1, k, Nk[d] // Nk[k]) for k in range(ds, d)]
        assert [(t, k, rows) for t, k, rows, _, _ in sk] == want
        assert all(w == 2 + 3 for _, _, _, w, _ in sk)
        offs = sorted(o for *_, o in sk)
        assert all(o % 256 == 0 for o in offs)
        N.lib().tt_plan_destroy(h)


def test_memory_footprint_follows_the_paper():
    """Sketch storage of PSTT2 is O(r n^floor(d/2)) and of PSTT2-onepass
    O(r n^ceil(d/2)) (Sec. 4.3, eqs. M_PSTT2 and M_PSTT2-onepass)."""
    n, r, p = 10, 3, 2
    for d in (5, 6, 7):
        for passes, expo in ((2, d // 2), (1, (d + 1) // 2)):
            st, h = plan([n] * d, ranks=[1] + [r] * (d - 1) + [1], p=p, passes=passes)
            biggest = max(rows for _, _, rows, _, _ in sketch_list(h))
            assert biggest == n ** expo
            N.lib().tt_plan_destroy(h)


def test_rank_clamping_and_padding():
    st, h = plan([4, 50, 3], ranks=[1, 9, 9, 1], p=2)
    assert st == N.TT_OK
    off, rp = layout(h)
    assert rp[:4] == [1, 4, 3, 1]  # min(N_k, M_k)
    assert off[1] == 0 and off[2] == 1 * 4 * 4 and off[3] == 16 + 4 * 50 * 3
    N.lib().tt_plan_destroy(h)
    st, h = plan([8, 8, 8, 8], eps=1e-6, rmax=6, p=10)
    off, rp = layout(h)
    assert rp[:5] == [1, 6, 6, 6, 1]
    N.lib().tt_plan_destroy(h)


@pytest.mark.parametrize("bad", [
    dict(dims=[5], ranks=[1, 1]),
    dict(dims=[5, 5], ranks=[2, 2, 1]),
    dict(dims=[5, 5], ranks=[1, 0, 1]),
    dict(dims=[5, 0, 5], ranks=[1, 1, 1, 1]),
    dict(dims=[5, 5], ranks=[1, 2, 1], p=0),
    dict(dims=[5, 5], ranks=[1, 2, 1], passes=3),
    dict(dims=[5, 5], eps=1e-3, rmax=0),
    dict(dims=[5, 5], eps=1e-3, rmax=60, p=10),
    dict(dims=[100, 100], ranks=[1, 70, 1]),
])
def test_invalid_problems_rejected(bad):
    dims = bad.pop("dims")
    st, h = plan(dims, **bad)
    assert st == N.TT_ERR_INVALID_ARG
    assert not h.value


def test_mixed_needs_fp32_storage():
    st, _ = plan([8, 8, 8], ranks=[1, 2, 2, 1], x_dtype=N.TT_F64, prec=N.TT_PREC_BF16)
    assert st == N.TT_ERR_UNSUPPORTED


def test_fp16_plans():
    """FP16 plans: FP32 storage only, a scale exponent within +-100, the same
    workspace as the BF16 plan of the shape (16-bit operands, same staging),
    and the scale kept in the stored problem."""
    st, _ = plan([8, 8, 8], ranks=[1, 2, 2, 1], x_dtype=N.TT_F64, prec=N.TT_PREC_FP16)
    assert st == N.TT_ERR_UNSUPPORTED
    for s in (-101, 101):
        st, h = plan([8, 8, 8], ranks=[1, 2, 2, 1], prec=N.TT_PREC_FP16, x_scale_log2=s)
        assert st == N.TT_ERR_INVALID_ARG and not h.value
    # other precisions ignore the field
    st, h = plan([8, 8, 8], ranks=[1, 2, 2, 1], prec=N.TT_PREC_BF16, x_scale_log2=500)
    assert st == N.TT_OK
    N.lib().tt_plan_destroy(h)
    for dims, kw in (([256, 256, 256, 256], dict(eps=1e-6, rmax=6, p=10)),
                     ([24] * 6, dict(eps=1e-6, rmax=16, p=10)),
                     ([40, 30, 50], dict(ranks=[1, 3, 4, 1], p=5))):
        st16, h16 = plan(dims, prec=N.TT_PREC_FP16, x_scale_log2=12, **kw)
        stbf, hbf = plan(dims, prec=N.TT_PREC_BF16, **kw)
        assert st16 == N.TT_OK and stbf == N.TT_OK
        assert sizes(h16)[1:] == sizes(hbf)[1:]
        # no tensor-core adjoint table for FP16 (its backward takes the SIMT adjoint)
        assert sizes(h16)[0] <= sizes(hbf)[0]
        assert N.lib().tt_sketch_kernel_kind(h16, dims[-1]) == N.lib().tt_sketch_kernel_kind(hbf, dims[-1])
        q = N.tt_problem()
        N.check(N.lib().tt_plan_problem(h16, 0, C.byref(q)), "problem")
        assert q.prec == N.TT_PREC_FP16 and q.x_scale_log2 == 12
        N.lib().tt_plan_destroy(h16)
        N.lib().tt_plan_destroy(hbf)
    # the 1 GiB slab of the 256^4 tensor runs on the tcgen05 slab kernel, both test-matrix kinds
    for flags in (0, N.TT_FLAG_KR):
        st, h = plan([256] * 4, eps=1e-6, rmax=6, p=10, prec=N.TT_PREC_FP16, x_scale_log2=16, flags=flags)
        assert st == N.TT_OK and N.lib().tt_sketch_kernel_kind(h, 16) == 2
        N.lib().tt_plan_destroy(h)


def test_status_strings():
    for s in range(10):
        assert N.lib().tt_status_string(s)
    assert b"ttsketch" in N.lib().tt_version()


def test_batched_plan_slices():
    probs = (N.tt_problem * 3)()
    for i, dims in enumerate([[4, 5, 6], [6, 6, 6, 6], [3, 9]]):
        probs[i] = N.make_problem(dims, ranks=[1] + [2] * (len(dims) - 1) + [1], p=2)
    h = C.c_void_p()
    N.check(N.lib().tt_sketch_plan_batched(probs, 3, C.byref(h)), "batched")
    _, ce, re_ = sizes(h)
    assert re_ == 4 + 5 + 3
    offs = [layout(h, i)[0] for i in range(3)]
    assert offs[1][1] == offs[0][3] + 2 * 6 * 1
    assert ce == offs[2][2] + 2 * 9 * 1
    N.lib().tt_plan_destroy(h)


def test_one_sided_plans_refuse_what_they_do_not_support():
    """TT_FLAG_ONESIDED: single-problem plans without TT_FLAG_DIFF (host-side
    checks, no device needed); the sketch list is every right sketch plus
    the left sketch of X_{d-1}."""
    import ctypes as C
    from paper_2111_10448_gb300 import _native as N
    L = N.lib()
    h = C.c_void_p()
    base = dict(ranks=[1, 2, 3, 2, 1], p=3, seed=1, x_dtype=N.TT_F32, prec=N.TT_PREC_FP64)
    ok = N.make_problem([6, 5, 4, 7], passes=1, flags=N.TT_FLAG_ONESIDED, **base)
    assert L.tt_sketch_plan(C.byref(ok), C.byref(h)) == N.TT_OK
    got = []
    for i in range(8):
        ty, k, w = C.c_int(), C.c_int(), C.c_int()
        rows, off = C.c_int64(), C.c_int64()
        if L.tt_plan_sketch_info(h, 0, i, C.byref(ty), C.byref(k), C.byref(rows), C.byref(w), C.byref(off)) != 0:
            break
        got.append((ty.value, k.value, rows.value, w.value))
    assert got == [(0, 1, 6, 5), (0, 2, 30, 6), (0, 3, 120, 5), (1, 3, 7, 5)]
    L.tt_plan_destroy(h)
    for kw in (dict(passes=1, flags=N.TT_FLAG_ONESIDED | N.TT_FLAG_DIFF),):
        bad = N.make_problem([6, 5, 4, 7], **kw, **base)
        assert L.tt_sketch_plan(C.byref(bad), C.byref(h)) == N.TT_ERR_UNSUPPORTED
    arr = (N.tt_problem * 2)(ok, ok)
    assert L.tt_sketch_plan_batched(arr, 2, C.byref(h)) == N.TT_ERR_UNSUPPORTED


def _staged_bytes(dims, sk, esz):
    """Staging tables of the generic tile kernel by the rule the plan states:
    column side keys w / wdiv over i_d, row side keys w % wdiv over i_1,
    staged when more than one tile would draw the rows; row-side tables over
    16 MiB need four column tiles of a plane; 256 MiB a table, 1 GiB an item."""
    d, n1, nd = len(dims), dims[0], dims[-1]
    Nk = [1]
    for v in dims:
        Nk.append(Nk[-1] * v)
    W = Nk[d - 1] // n1
    tiles_a, tiles_b = -(-n1 // 64), -(-nd // 32)
    total = 0
    for ty, k, rows, width, _ in sk:
        lpad = -(-width // 16) * 16
        wdiv = Nk[k] // n1
        tb = 0
        if ty == 0 and wdiv * tiles_a >= 2:
            tb = (W // wdiv) * nd * lpad * esz
        if ty == 1 and (W // wdiv) * tiles_b >= 2:
            tb = wdiv * n1 * lpad * esz
            if tiles_b < 4 and tb > 16 << 20:
                tb = 0
        if 0 < tb <= 256 << 20 and total + tb <= 1 << 30:
            total += -(-tb // 256) * 256
    return total


@pytest.mark.parametrize("dims,r", [([200] * 4, [1, 40, 40, 40, 1]), ([960] * 3, [1, 25, 25, 1]),
                                    ([96] * 5, [1, 17, 18, 18, 17, 1]), ([70, 3, 5, 45], [1, 4, 5, 4, 1]),
                                    ([48, 40, 36, 40, 64], [1, 20, 30, 30, 20, 1]),
                                    ([100] * 4, [1, 40, 40, 40, 1])])
def test_generic_kernel_staging_tables_follow_their_rule(dims, r):
    """The BF16 / TF32 workspace of a shape on the generic tile kernel exceeds
    the FP64 one by exactly its staged test-matrix rows (2 or 4 bytes an
    entry), capped per sketch and per item."""
    ws = {}
    for prec in (N.TT_PREC_FP64, N.TT_PREC_BF16, N.TT_PREC_TF32):
        st, h = plan(dims, ranks=r, p=10, x_dtype=N.TT_F32, prec=prec)
        assert st == N.TT_OK
        ws[prec] = sizes(h)[0]
        if prec == N.TT_PREC_BF16:
            sk = sketch_list(h)
            assert N.lib().tt_sketch_kernel_kind(h, dims[-1]) == 1
        N.lib().tt_plan_destroy(h)
    assert ws[N.TT_PREC_BF16] - ws[N.TT_PREC_FP64] == _staged_bytes(dims, sk, 2)
    assert ws[N.TT_PREC_TF32] - ws[N.TT_PREC_FP64] == _staged_bytes(dims, sk, 4)
    assert ws[N.TT_PREC_TF32] - ws[N.TT_PREC_FP64] <= 1 << 30


def test_readme_c_example_compiles_and_links(tmp_path):
    """The C quick start of the README compiles warning-free against
    include/ttsketch.h and links against the built library."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if gcc is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("gcc or the CUDA headers are not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "README.md")).read()
    m = re.search(r"## Quick start \(C\)\s*```c\n(.*?)```", text, re.S)
    assert m, "no C quick start in the README"
    src = tmp_path / "app.c"
    src.write_text(m.group(1))
    N.lib()  # the library is built
    libdir = os.path.dirname(N.LIB_PATH)
    cudalib = next((p for p in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib")) if os.path.isdir(p)), None)
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
           "-I", os.path.join(cuda, "include"), str(src), "-L", libdir, "-lttsketch"]
    if cudalib:
        cmd += ["-L", cudalib]
    cmd += ["-lcudart", "-o", str(tmp_path / "app")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_device_calls_check_their_arguments_on_the_host():
    """Argument errors of the generator, test-matrix and Tucker calls come back
    synchronously as TT_ERR_INVALID_ARG before anything is launched, and empty
    ranges are TT_OK without a launch (no device needed for either)."""
    L = N.lib()
    BAD, OK = N.TT_ERR_INVALID_ARG, N.TT_OK
    dummy = C.c_void_p(256)  # never dereferenced: every case returns before a launch
    null = C.c_void_p(None)
    n3 = (C.c_int64 * 3)(4, 5, 6)
    n0 = (C.c_int64 * 3)(4, 0, 6)
    # test matrix
    assert L.tt_test_matrix(1, 0, 0, 10, 4, N.TT_PREC_BF16, null, null) == BAD
    assert L.tt_test_matrix(1, 0, 0, -1, 4, N.TT_PREC_BF16, dummy, null) == BAD
    assert L.tt_test_matrix(1, 0, -3, 10, 4, N.TT_PREC_BF16, dummy, null) == BAD
    assert L.tt_test_matrix(1, 0, 0, 10, N.TT_MAXL + 1, N.TT_PREC_BF16, dummy, null) == BAD
    assert L.tt_test_matrix(1, 0, 0, 10, 4, 7, dummy, null) == BAD
    assert L.tt_test_matrix(1, 0, 0, 0, 4, N.TT_PREC_BF16, dummy, null) == OK
    assert L.tt_test_matrix(1, 0, 0, 0, 4, N.TT_PREC_FP16, dummy, null) == OK
    # FP16 scale helper: null pointers, negative count, unknown dtype; empty is s = 0
    sv = C.c_int(7)
    assert L.tt_x_scale_log2(null, N.TT_F32, 4, C.byref(sv), null) == BAD
    assert L.tt_x_scale_log2(dummy, N.TT_F32, 4, None, null) == BAD
    assert L.tt_x_scale_log2(dummy, N.TT_F32, -1, C.byref(sv), null) == BAD
    assert L.tt_x_scale_log2(dummy, 5, 4, C.byref(sv), null) == BAD
    assert L.tt_x_scale_log2(dummy, N.TT_F32, 0, C.byref(sv), null) == OK and sv.value == 0
    # raw Philox
    assert L.tt_philox4x32_10(null, 1, 2, dummy, 4, null) == BAD
    assert L.tt_philox4x32_10(dummy, 1, 2, dummy, -1, null) == BAD
    assert L.tt_philox4x32_10(dummy, 1, 2, dummy, 0, null) == OK
    # generators: bad order, zero mode, slab outside the last mode, dtype, empty slab
    for gen in (L.tt_generate_hilbert, L.tt_generate_hilbert_type):
        assert gen(0, n3, 0, 1, dummy, N.TT_F32, null) == BAD
        assert gen(N.TT_MAXD + 1, n3, 0, 1, dummy, N.TT_F32, null) == BAD
        assert gen(3, n0, 0, 1, dummy, N.TT_F32, null) == BAD
        assert gen(3, n3, 4, 3, dummy, N.TT_F32, null) == BAD
        assert gen(3, n3, 0, 1, null, N.TT_F32, null) == BAD
        assert gen(3, n3, 0, 1, dummy, 5, null) == BAD
        assert gen(3, n3, 6, 0, dummy, N.TT_F32, null) == OK
    cen = (C.c_double * 6)(0.0, 0.1, 0.2, 0.3, 0.4, 0.5)
    bumps = L.tt_generate_gaussian_bumps
    assert bumps(3, n3, 0, 10.0, cen, 0, 1, dummy, N.TT_F32, null) == BAD          # no bumps
    assert bumps(3, n3, 2, float("nan"), cen, 0, 1, dummy, N.TT_F32, null) == BAD  # gamma
    assert bumps(3, n3, 2, -1.0, cen, 0, 1, dummy, N.TT_F32, null) == BAD
    assert bumps(3, n3, 2, 10.0, null, 0, 1, dummy, N.TT_F32, null) == BAD         # centres
    assert bumps(3, n3, 2, 10.0, cen, 5, 2, dummy, N.TT_F32, null) == BAD          # slab outside
    assert bumps(3, n3, 2, 10.0, cen, 0, 0, dummy, N.TT_F32, null) == OK
    # Tucker steps
    assert L.tt_core_mode2(null, 2, 3, 2, dummy, 5, dummy, null) == BAD
    assert L.tt_core_mode2(dummy, 0, 3, 2, dummy, 5, dummy, null) == BAD
    assert L.tt_core_mode2(dummy, 2, 3, 2, dummy, 0, dummy, null) == BAD
    assert L.tt_swap12(dummy, 2, 3, 4, dummy, null) == BAD                         # in == out
    assert L.tt_swap12(dummy, 0, 3, 4, C.c_void_p(512), null) == BAD


def test_batched_plans_stage_no_generic_rows():
    """The batched sketch kernel draws its test-matrix rows per tile, so a
    batched plan reserves no staging tables: its BF16 / TF32 workspace equals
    the FP64 one for shapes outside the plane and small-plane kernels."""
    probs = [([70, 3, 5, 45], [1, 4, 5, 4, 1]), ([200] * 3, [1, 20, 20, 1])]

    def ws_of(prec):
        arr = (N.tt_problem * len(probs))(*[N.make_problem(d, ranks=r, p=10, x_dtype=N.TT_F32, prec=prec)
                                             for d, r in probs])
        h = C.c_void_p()
        assert N.lib().tt_sketch_plan_batched(arr, len(probs), C.byref(h)) == N.TT_OK
        w = sizes(h)[0]
        N.lib().tt_plan_destroy(h)
        return w

    assert ws_of(N.TT_PREC_BF16) == ws_of(N.TT_PREC_FP64) == ws_of(N.TT_PREC_TF32)


def test_khatri_rao_plans():
    """TT_FLAG_KR: single-problem plans only; the workspace grows by the staged
    factors (sum over sketches of the factor sizes of their modes)."""
    L = N.lib()
    base = N.make_problem([16] * 4, ranks=[1, 4, 4, 4, 1], p=5, seed=1)
    krq = N.make_problem([16] * 4, ranks=[1, 4, 4, 4, 1], p=5, seed=1, flags=N.TT_FLAG_KR)
    sizes = []
    for q in (base, krq):
        h = C.c_void_p()
        N.check(L.tt_sketch_plan(C.byref(q), C.byref(h)), "plan")
        ws = C.c_size_t()
        N.check(L.tt_plan_sizes(h, C.byref(ws), None, None), "sizes")
        sizes.append(ws.value)
        L.tt_plan_destroy(h)
    # S_1: modes 2..4, S_2: 3..4, R_2: 1..2, R_3: 1..3; width 9, factor rows of 16
    factors = (3 + 2 + 2 + 3) * 16 * 16 * 8
    assert factors <= sizes[1] - sizes[0] <= factors + 4 * 256
    arr = (N.tt_problem * 2)(krq, krq)
    h = C.c_void_p()
    assert L.tt_sketch_plan_batched(arr, 2, C.byref(h)) == N.TT_ERR_UNSUPPORTED


def test_stream_state_checks_on_the_host():
    """Checkpoint calls: size of the state (header + slab bitmap + every sketch
    in FP64), refusal for batched and two-pass plans, argument and state errors
    before any device work (no stream is open on a fresh plan)."""
    L = N.lib()
    st, h = plan([40, 7, 6, 70], ranks=[1, 4, 5, 4, 1], p=6)
    assert st == N.TT_OK
    n = C.c_size_t()
    N.check(L.tt_pstt2_state_size(h, C.byref(n)), "size")
    sk = sketch_list(h)
    assert n.value == 272 + 72 + 8 * sum(rows * w for _, _, rows, w, _ in sk)
    dummy, null = C.c_void_p(256), C.c_void_p(None)
    buf = (C.c_ubyte * n.value)()
    assert L.tt_pstt2_state_size(h, None) == N.TT_ERR_INVALID_ARG
    assert L.tt_pstt2_export_state(h, dummy, buf, n.value - 1, null) == N.TT_ERR_INVALID_ARG
    assert L.tt_pstt2_export_state(h, null, buf, n.value, null) == N.TT_ERR_INVALID_ARG
    assert L.tt_pstt2_export_state(h, dummy, buf, n.value, null) == N.TT_ERR_STATE      # nothing begun
    assert L.tt_pstt2_import_state(h, dummy, buf, n.value - 1, null) == N.TT_ERR_INVALID_ARG
    assert L.tt_pstt2_import_state(h, dummy, buf, n.value, null) == N.TT_ERR_INVALID_ARG  # no header
    L.tt_plan_destroy(h)
    st, h2 = plan([40, 7, 6, 70], ranks=[1, 4, 5, 4, 1], p=6, passes=2)
    assert L.tt_pstt2_state_size(h2, C.byref(n)) == N.TT_ERR_UNSUPPORTED
    L.tt_plan_destroy(h2)


def test_tt_log_prints_plan_layouts(tmp_path):
    """TT_LOG=1: one stderr line per plan item and one for the plan (host only)."""
    import subprocess
    import sys
    code = ("import ctypes as C; from paper_2111_10448_gb300 import _native as N; "
            "q = N.make_problem([64, 8, 8, 64], eps=1e-6, rmax=6, p=10, prec=N.TT_PREC_FP16, x_scale_log2=3); "
            "h = C.c_void_p(); N.check(N.lib().tt_sketch_plan(C.byref(q), C.byref(h)), 'plan'); "
            "N.lib().tt_plan_destroy(h)")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, TT_LOG="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "ttsketch: plan" in r.stderr and "64x8x8x64 fp16" in r.stderr, r.stderr
    env["TT_LOG"] = "0"
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "ttsketch:" not in r.stderr

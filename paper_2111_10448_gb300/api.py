"""Python wrapper of one plan: device buffers as torch tensors, calls through
the C ABI (argument marshalling only)."""
import ctypes as C

import torch

from . import _native as N

_DT = {torch.float32: N.TT_F32, torch.float64: N.TT_F64}


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class TTSketch:
    """One decomposition problem (or a batch of them) with its device state.

    dims: mode sizes; ranks (fixed-rank mode, [1, r_1, .., r_{d-1}, 1]) or eps
    (> 0, tolerance mode, with rmax); p: oversampling; seed: Philox key;
    passes: 1 (one-pass, the hot path) or 2; x_dtype: torch.float32/float64;
    prec: 'fp64' | 'tf32' | 'bf16' | 'fp16'; x_scale_log2: the power-of-two
    scale s of X before an FP16 split (X 2^s must stay below 65520; see
    x_scale_log2() below); short_chains: TT_FLAG_SHORT_CHAINS (shorter FP32
    accumulation chains in the tcgen05 kernels); one_sided: the one-sided PSTT-onepass
    (every unfolding sketched from the right, last core by least squares)
    instead of the two-sided PSTT2-onepass; drm: 'gauss' (dense Gaussian test
    matrices) or 'kr' (Khatri-Rao products of per-mode Gaussian factors).
    """

    PRECS = {"fp64": N.TT_PREC_FP64, "tf32": N.TT_PREC_TF32, "bf16": N.TT_PREC_BF16,
             "fp16": N.TT_PREC_FP16}

    def __init__(self, dims, *, ranks=None, eps=0.0, rmax=0, p=5, seed=1, passes=1,
                 x_dtype=torch.float32, prec="fp64", device="cuda", batch=None, diff=False,
                 one_sided=False, drm="gauss", x_scale_log2=0, short_chains=False):
        L = N.lib()
        self.device = torch.device(device)
        if batch is None:
            probs = [dict(dims=dims, ranks=ranks, eps=eps, rmax=rmax, p=p, seed=seed)]
        else:
            probs = batch
        arr = (N.tt_problem * len(probs))()
        for i, pr in enumerate(probs):
            arr[i] = N.make_problem(pr["dims"], ranks=pr.get("ranks"), eps=pr.get("eps", eps),
                                    rmax=pr.get("rmax", rmax), p=pr.get("p", p),
                                    seed=pr.get("seed", seed), passes=passes,
                                    x_dtype=_DT[x_dtype], prec=self.PRECS[prec],
                                    flags=(N.TT_FLAG_DIFF if diff else 0) |
                                    (N.TT_FLAG_ONESIDED if one_sided else 0) |
                                    (N.TT_FLAG_KR if drm == "kr" else 0) |
                                    (N.TT_FLAG_SHORT_CHAINS if short_chains else 0),
                                    x_scale_log2=pr.get("x_scale_log2", x_scale_log2))
        h = C.c_void_p()
        if batch is None:
            N.check(L.tt_sketch_plan(C.byref(arr[0]), C.byref(h)), "tt_sketch_plan")
        else:
            N.check(L.tt_sketch_plan_batched(arr, len(probs), C.byref(h)), "tt_sketch_plan_batched")
        self.plan = h
        self.count = len(probs)
        self.x_dtype = x_dtype
        ws, ce, re_ = C.c_size_t(), C.c_int64(), C.c_int()
        N.check(L.tt_plan_sizes(h, C.byref(ws), C.byref(ce), C.byref(re_)), "tt_plan_sizes")
        self.ws_bytes, self.core_entries, self.rank_entries = ws.value, ce.value, re_.value
        self.items = []
        for i in range(self.count):
            off = (C.c_int64 * (N.TT_MAXD + 1))()
            rp = (C.c_int * (N.TT_MAXD + 1))()
            N.check(L.tt_plan_core_layout(h, i, off, rp), "tt_plan_core_layout")
            q = N.tt_problem()
            N.check(L.tt_plan_problem(h, i, C.byref(q)), "tt_plan_problem")
            d = q.d
            self.items.append(dict(d=d, dims=[q.n[k] for k in range(d)],
                                   core_off=[off[k] for k in range(d + 1)],
                                   rpad=[rp[k] for k in range(d + 1)]))
        self.dims = self.items[0]["dims"]
        self.d = self.items[0]["d"]
        self.ws = torch.empty(max(self.ws_bytes, 8) // 8 + 32, dtype=torch.float64, device=self.device)
        self.cores = torch.zeros(max(self.core_entries, 1), dtype=torch.float64, device=self.device)
        self.ranks = torch.zeros(max(self.rank_entries, 1), dtype=torch.int32, device=self.device)

    def __del__(self):
        try:
            if getattr(self, "plan", None):
                N.lib().tt_plan_destroy(self.plan)
                self.plan = None
        except Exception:
            pass

    # --------------------------------------------------------------- forward
    def pstt2(self, X, stream=None):
        N.check(N.lib().tt_pstt2(self.plan, _ptr(X), _ptr(self.ws), _ptr(self.cores), _ptr(self.ranks),
                                 _stream(stream)), "tt_pstt2")
        return self

    def begin(self, stream=None):
        N.check(N.lib().tt_pstt2_begin(self.plan, _ptr(self.ws), _stream(stream)), "tt_pstt2_begin")

    def accumulate(self, slab, first, count, stream=None):
        N.check(N.lib().tt_pstt2_accumulate(self.plan, _ptr(slab), int(first), int(count), _ptr(self.ws),
                                            _stream(stream)), "tt_pstt2_accumulate")

    def export_state(self, stream=None):
        """The state of the stream in progress (sketches, slabs added) as a
        host uint8 array; resume it with import_state on any TTSketch of the
        same problem."""
        import numpy as np
        n = C.c_size_t()
        N.check(N.lib().tt_pstt2_state_size(self.plan, C.byref(n)), "tt_pstt2_state_size")
        buf = np.empty(n.value, dtype=np.uint8)
        N.check(N.lib().tt_pstt2_export_state(self.plan, _ptr(self.ws), C.c_void_p(buf.ctypes.data), n.value,
                                              _stream(stream)), "tt_pstt2_export_state")
        return buf

    def import_state(self, buf, stream=None):
        """Open a stream from an exported state (instead of begin)."""
        import numpy as np
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        N.check(N.lib().tt_pstt2_import_state(self.plan, _ptr(self.ws), C.c_void_p(buf.ctypes.data), buf.size,
                                              _stream(stream)), "tt_pstt2_import_state")

    def finalize(self, stream=None):
        N.check(N.lib().tt_pstt2_finalize(self.plan, _ptr(self.ws), _ptr(self.cores), _ptr(self.ranks),
                                          _stream(stream)), "tt_pstt2_finalize")
        return self

    def batched(self, Xs, stream=None):
        arr = (C.c_void_p * len(Xs))(*[x.data_ptr() for x in Xs])
        N.check(N.lib().tt_pstt2_batched(self.plan, arr, _ptr(self.ws), _ptr(self.cores), _ptr(self.ranks),
                                         _stream(stream)), "tt_pstt2_batched")
        return self

    def batch_config(self, ta=64, chunk=4, ctas_per_sm=4):
        N.check(N.lib().tt_plan_batch_config(self.plan, int(ta), int(chunk), int(ctas_per_sm)),
                "tt_plan_batch_config")

    def autotune(self, Xs, stream=None):
        """Pick the batched sketch launch shape by timing the candidates on Xs;
        returns (ta, chunk, ctas_per_sm).  Leaves a valid decomposition."""
        arr = (C.c_void_p * len(Xs))(*[x.data_ptr() for x in Xs])
        best = (C.c_int * 3)()
        N.check(N.lib().tt_plan_autotune(self.plan, arr, _ptr(self.ws), _ptr(self.cores), _ptr(self.ranks),
                                         _stream(stream), best), "tt_plan_autotune")
        return tuple(best)

    def backward(self, dcores, dX, stream=None):
        N.check(N.lib().tt_pstt2_backward(self.plan, _ptr(self.ws), _ptr(dcores), _ptr(dX), _stream(stream)),
                "tt_pstt2_backward")

    # -------------------------------------------------------- reconstruction
    def reconstruct(self, dtype=torch.float64, cores=None, stream=None):
        n = 1
        for v in self.dims:
            n *= v
        out = torch.empty(n, dtype=dtype, device=self.device)
        N.check(N.lib().tt_reconstruct(self.plan, _ptr(self.cores if cores is None else cores), _ptr(out),
                                       _DT[dtype], _ptr(self.ws), _stream(stream)), "tt_reconstruct")
        return out

    def error(self, X, stream=None, cores=None):
        out2 = torch.empty(2, dtype=torch.float64, device=self.device)
        N.check(N.lib().tt_reconstruct_error(self.plan, _ptr(self.cores if cores is None else cores), _ptr(X),
                                             _ptr(out2), _ptr(self.ws), _stream(stream)),
                "tt_reconstruct_error")
        return out2

    def reconstruct_backward(self, dXt, cores=None, stream=None):
        dc = torch.empty_like(self.cores)
        N.check(N.lib().tt_reconstruct_backward(self.plan, _ptr(self.cores if cores is None else cores), _ptr(dXt),
                                                _DT[dXt.dtype], _ptr(dc), _ptr(self.ws), _stream(stream)),
                "tt_reconstruct_backward")
        return dc

    def sketches(self, item=0, stream=None):
        """Every sketch of one item, read from the workspace: list of
        (type, k, tensor rows x width) -- valid between accumulate and finalize."""
        N.check(N.lib().tt_pstt2_sync(self.plan, _ptr(self.ws), _stream(stream)), "tt_pstt2_sync")
        out = []
        i = 0
        while True:
            ty, k, w = C.c_int(), C.c_int(), C.c_int()
            rows, off = C.c_int64(), C.c_int64()
            st = N.lib().tt_plan_sketch_info(self.plan, item, i, C.byref(ty), C.byref(k), C.byref(rows),
                                             C.byref(w), C.byref(off))
            if st != N.TT_OK:
                break
            flat = self.ws[off.value // 8: off.value // 8 + rows.value * w.value]
            out.append((ty.value, k.value, flat.reshape(w.value, rows.value).T))
            i += 1
        return out

    def kernel_kind(self, count_last=None):
        """0 = FP64 SIMT, 1 = generic tensor-core (mma.sync), 2 = tcgen05 plane kernel,
        3 = small-plane tensor-core kernel."""
        c = self.dims[-1] if count_last is None else count_last
        return N.lib().tt_sketch_kernel_kind(self.plan, int(c))

    # ---------------------------------------------------------------- status
    def status(self, stream=None):
        st = C.c_int()
        rk = (C.c_int * max(self.rank_entries, 1))()
        N.check(N.lib().tt_query_status(self.plan, _ptr(self.ws), _ptr(self.ranks), C.byref(st), rk,
                                        _stream(stream)), "tt_query_status")
        return st.value, list(rk)[:self.rank_entries]

    def core_list(self, item=0):
        """Cores of one item as host float64 arrays of shape (r_{k-1}, n_k, r_k)
        (actual ranks, padding removed)."""
        import numpy as np
        it = self.items[item]
        _, ranks = self.status()
        base = sum(self.items[i]["d"] + 1 for i in range(item))
        r = ranks[base:base + it["d"] + 1]
        host = self.cores.cpu().numpy()
        out = []
        for k in range(1, it["d"] + 1):
            rp0, rp1, n = it["rpad"][k - 1], it["rpad"][k], it["dims"][k - 1]
            G = host[it["core_off"][k]:it["core_off"][k] + rp0 * n * rp1].reshape((rp0, n, rp1), order="F")
            out.append(np.ascontiguousarray(G[:r[k - 1], :, :r[k]]))
        return out


class PSTT2Fn(torch.autograd.Function):
    """X -> padded TT cores (one-pass PSTT2) with the hand-written adjoint
    (tt_pstt2_backward): pivots and ranks are frozen at this forward call."""

    @staticmethod
    def forward(ctx, X, sk):
        sk.pstt2(X.detach().contiguous())
        ctx.sk = sk
        ctx.xshape = X.shape
        return sk.cores.clone()

    @staticmethod
    def backward(ctx, dcores):
        sk = ctx.sk
        dX = torch.empty(ctx.xshape, dtype=sk.x_dtype, device=sk.device)
        sk.backward(dcores.contiguous(), dX)
        return dX, None


class TTReconstructFn(torch.autograd.Function):
    """padded TT cores -> dense X~ with its adjoint (tt_reconstruct_backward)."""

    @staticmethod
    def forward(ctx, cores, sk, dtype):
        ctx.sk = sk
        ctx.save_for_backward(cores)
        return sk.reconstruct(dtype, cores=cores.detach().contiguous())

    @staticmethod
    def backward(ctx, dXt):
        (cores,) = ctx.saved_tensors
        return ctx.sk.reconstruct_backward(dXt.contiguous(), cores=cores.contiguous()), None, None


def x_scale_log2(X, stream=None):
    """The FP16 scale exponent of tt_x_scale_log2 for the device tensor X
    (one reduction kernel over X; waits for it)."""
    s = C.c_int(0)
    N.check(N.lib().tt_x_scale_log2(_ptr(X), _DT[X.dtype], X.numel(), C.byref(s), _stream(stream)),
            "tt_x_scale_log2")
    return s.value


def pstt2(X, dims, **kw):
    """One-shot convenience: returns the TTSketch holding the cores."""
    t = TTSketch(dims, x_dtype=X.dtype, **kw)
    return t.pstt2(X)


def tucker2tt(G, factors, *, prec="fp64", stream=None, **kw):
    """Tucker2TT (Algorithm 3): TT cores of X = G x_1 A_1 ... x_d A_d without
    forming X.  G: the Tucker core on the device (column-major flat, dims
    [A.shape[1] for A in factors]); factors: device tensors A_k of shape
    (n_k, s_k) with orthonormal columns; kw: the TTSketch arguments of the
    decomposition of G (ranks or eps/rmax, p, seed, passes, ...).  Returns
    (cores, sketch): cores[k] is a device float64 tensor of shape
    (rpad_{k-1}, n_k, rpad_k) (column-major; rows and columns past the ranks
    are zero), sketch the TTSketch of G (ranks: sketch.status()[1])."""
    s = [int(A.shape[1]) for A in factors]
    t = TTSketch(s, x_dtype=G.dtype, prec=prec, device=G.device, **kw).pstt2(G, stream)
    it = t.items[0]
    out = []
    for k, A in enumerate(factors, start=1):
        n = int(A.shape[0])
        rp0, rp1 = it["rpad"][k - 1], it["rpad"][k]
        Acm = A.to(torch.float64).t().contiguous()  # column-major n x s
        H = t.cores[it["core_off"][k]:it["core_off"][k] + rp0 * s[k - 1] * rp1]
        T = torch.empty(rp0 * n * rp1, dtype=torch.float64, device=G.device)
        N.check(N.lib().tt_core_mode2(_ptr(H), rp0, s[k - 1], rp1, _ptr(Acm), n, _ptr(T), _stream(stream)),
                "tt_core_mode2")
        out.append(T.view(rp1, n, rp0).permute(2, 1, 0))
    return out, t


def tt2tucker(cores, tranks, *, p=5, seed=1, stream=None):
    """TT2Tucker (Algorithm 4): an orthogonal Tucker format of the TT tensor
    with the given cores.  cores: device float64 tensors T_k of shape
    (r_{k-1}, n_k, r_k) (contiguous in the column-major sense: T.permute(2, 1,
    0) contiguous, as tucker2tt returns them, or plain row-major tensors of that
    shape, which are converted); tranks: the multilinear target ranks t_k.
    Step 2 for core k is the one-sided two-pass PSTT (d = 2) of the mode-2
    matricization (T_k)_(2) with target rank t_k, test-matrix key seed + k:
    A_k is its first core, H_k its second, folded back.  Returns (H, A): H[k]
    of shape (r_{k-1}, tpad_k, r_k) and A[k] of shape (n_k, tpad_k), both
    device float64 (columns past the found rank zero)."""
    Hs, As = [], []
    for k, T in enumerate(cores, start=1):
        r0, n, r1 = (int(v) for v in T.shape)
        Tcm = T.to(torch.float64).permute(2, 1, 0).contiguous()  # column-major r0 x n x r1
        M = torch.empty(n * r0 * r1, dtype=torch.float64, device=Tcm.device)
        N.check(N.lib().tt_swap12(_ptr(Tcm), r0, n, r1, _ptr(M), _stream(stream)), "tt_swap12")
        t = min(int(tranks[k - 1]), n, r0 * r1)
        sk = TTSketch([n, r0 * r1], ranks=[1, t, 1], p=p, seed=seed + k, passes=2, one_sided=True,
                      x_dtype=torch.float64, prec="fp64", device=Tcm.device).pstt2(M, stream)
        it = sk.items[0]
        tp = it["rpad"][1]
        A = sk.cores[it["core_off"][1]:it["core_off"][1] + n * tp].view(tp, n).t()      # n x tp
        H2 = sk.cores[it["core_off"][2]:it["core_off"][2] + tp * r0 * r1]               # tp x (r0 r1), column-major
        H = torch.empty(r0 * tp * r1, dtype=torch.float64, device=Tcm.device)
        N.check(N.lib().tt_swap12(_ptr(H2), tp, r0, r1, _ptr(H), _stream(stream)), "tt_swap12")
        Hs.append(H.view(r1, tp, r0).permute(2, 1, 0))
        As.append(A.clone())
    return Hs, As

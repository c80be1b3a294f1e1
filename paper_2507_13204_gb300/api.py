"""Problem objects over the C ABI (argument marshalling only).

A Problem keeps the tensors it lent to kg_create alive for as long as the
handle exists, allocates output tensors with torch on the problem's device and
calls the library.  No arithmetic of the method happens here.
"""
from __future__ import annotations

import torch

from . import _lib as L

_DT = {torch.float64: L.KG_F64, torch.float32: L.KG_F32}
STRATEGIES = {"auto": L.KG_STRATEGY_AUTO, "atomic": L.KG_STRATEGY_ATOMIC, "csr": L.KG_STRATEGY_CSR,
              "transpose": L.KG_STRATEGY_TRANSPOSE, "fused": L.KG_STRATEGY_FUSED,
              "shared": L.KG_STRATEGY_SHARED, "warp": L.KG_STRATEGY_WARP, "tile": L.KG_STRATEGY_TILE}
MODES = {"auto": L.KG_MODE_AUTO, "recompute": L.KG_MODE_RECOMPUTE, "tape": L.KG_MODE_TAPE}
ARITHS = {"auto": L.KG_ARITH_AUTO, "native": L.KG_ARITH_NATIVE, "pair": L.KG_ARITH_PAIR}


def _dev_tensor(t: torch.Tensor, dtype=None) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError("kg: problem data must be CUDA tensors")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"kg: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("kg: tensors must be contiguous")
    return t


def _arg(t, n: int, dtype, device, what: str, host: bool = False):
    """A tensor the library reads or writes n elements of.  Checked here, so that a wrong
    device, dtype, layout or length raises before any copy or kernel touches it (four
    cheap queries on the fast path; the message is built only on failure)."""
    if t is None:
        return None
    if (not isinstance(t, torch.Tensor) or t.dtype is not dtype or t.numel() != n
            or not t.is_contiguous() or (t.is_cuda if host else t.device != device)):
        _arg_error(t, n, dtype, device, what, host)
    return t


def _arg_error(t, n, dtype, device, what, host):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"kg: {what} must be a torch.Tensor")
    if host and t.is_cuda:
        raise ValueError(f"kg: {what} must be a host tensor")
    if not host and t.device != device:
        raise ValueError(f"kg: {what} must be a CUDA tensor on {device}")
    if t.dtype != dtype:
        raise ValueError(f"kg: {what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"kg: {what} must be contiguous")
    raise ValueError(f"kg: {what} must have {n} elements, has {t.numel()}")


class Problem:
    kind = 0

    def __init__(self, sizes, data, dtype: torch.dtype, strategy="auto", mode="auto",
                 arith="auto", check=False, block=0, team=0, tile=0, tape_budget_bytes=0,
                 stream=None):
        self.dtype = dtype
        self.device = data[0].device
        self._data = list(data)  # borrowed by the library: keep alive
        opt = L.options(dtype=_DT[dtype], strategy=STRATEGIES[strategy], mode=MODES[mode],
                        arith=ARITHS[arith], check=int(bool(check)), block=block, team=team,
                        tile=tile, tape_budget_bytes=tape_budget_bytes)
        with torch.cuda.device(self.device):
            self.handle = L.kg_create(self.kind, sizes, self._data, opt, stream)
        self.sizes = tuple(int(s) for s in sizes)

    # -- lifetime
    def close(self):
        if getattr(self, "handle", None):
            L.kg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- shapes
    @property
    def nx(self) -> int:
        raise NotImplementedError

    @property
    def ndata(self) -> int:
        """Length of gdata, the gradient w.r.t. the first data operand (0: not offered)."""
        return 0

    def _vec(self, t, what, host=False):
        return _arg(t, self.nx, self.dtype, self.device, what, host)

    def _one(self, t, what, host=False):
        return _arg(t, 1, self.dtype, self.device, what, host)

    def _scalar(self):
        return torch.empty((), dtype=self.dtype, device=self.device)

    # -- calls
    def eval(self, x, f=None, stream=None):
        f = self._scalar() if f is None else self._one(f, "f")
        L.kg_eval(self.handle, self._vec(x, "x"), f, stream)
        return f

    def grad(self, x, gx=None, f=None, gdata=None, seed=None, accumulate=False, stream=None):
        gx = torch.empty(self.nx, dtype=self.dtype, device=self.device) if gx is None else self._vec(gx, "gx")
        f = self._scalar() if f is None else self._one(f, "f")
        if gdata is not None:
            if not self.ndata:
                raise ValueError("kg: this kind offers no gradient w.r.t. its data (gdata)")
            _arg(gdata, self.ndata, self.dtype, self.device, "gdata")
        L.kg_grad(self.handle, self._vec(x, "x"), f, gx, gdata, self._one(seed, "seed"),
                  int(accumulate), stream)
        return f, gx

    def hvp(self, x, v, hv=None, seed=None, accumulate=False, stream=None):
        """Hessian-vector product fbar * H(x) v (x may be None for the quadratic kinds)."""
        hv = torch.empty(self.nx, dtype=self.dtype, device=self.device) if hv is None else self._vec(hv, "hv")
        L.kg_hvp(self.handle, self._vec(x, "x"), self._vec(v, "v"), hv, self._one(seed, "seed"),
                 int(accumulate), stream)
        return hv

    def eval_tape(self, x, f=None, stream=None):
        """Forward pass that records the problem's tape (TAPE mode)."""
        f = self._scalar() if f is None else self._one(f, "f")
        L.kg_eval_tape(self.handle, self._vec(x, "x"), f, stream)
        return f

    @property
    def tape_generation(self) -> int:
        """Count of launches so far that wrote the tape (kg_tape_generation)."""
        return L.kg_tape_generation(self.handle)

    def grad_from_tape(self, gx=None, seed=None, accumulate=False, stream=None):
        """Reverse pass from the tape as the last call that wrote it left it."""
        gx = torch.empty(self.nx, dtype=self.dtype, device=self.device) if gx is None else self._vec(gx, "gx")
        L.kg_grad_from_tape(self.handle, gx, self._one(seed, "seed"), int(accumulate), stream)
        return gx

    def grad_host(self, x_host, gx_host, f_host=None, stream=None):
        """kg_grad on host buffers (pinned for overlap): the library copies x in and
        gx (and f) out."""
        L.kg_grad_host(self.handle, self._vec(x_host, "x_host", host=True),
                       self._one(f_host, "f_host", host=True), self._vec(gx_host, "gx_host", host=True),
                       stream)

    def sync(self):
        L.kg_sync(self.handle)

    @property
    def config(self):
        """Resolved (strategy, mode, arith)."""
        return L.kg_get_config(self.handle)

    @property
    def workspace_bytes(self) -> int:
        return L.kg_workspace_bytes(self.handle)


class QuadForm(Problem):
    """f(x) = ||A x||^2, A (m x n) row-major on the device."""
    kind = L.KG_QUADFORM

    def __init__(self, A: torch.Tensor, **kw):
        A = _dev_tensor(A)
        m, n = A.shape
        super().__init__([m, n], [A], A.dtype, **kw)
        self.m, self.n = m, n

    @property
    def nx(self):
        return self.n

    @property
    def ndata(self):
        return self.m * self.n


class SpQuadForm(Problem):
    """f(x) = ||A x||^2, A (m x n) sparse in compressed sparse rows on the device:
    rowptr int32 [m + 1], col int32 [nnz], val [nnz].  gdata of grad() is the
    gradient w.r.t. val."""
    kind = L.KG_SPQUADFORM

    def __init__(self, rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, n: int, **kw):
        rowptr = _dev_tensor(rowptr, torch.int32)
        col = _dev_tensor(col, torch.int32)
        val = _dev_tensor(val)
        if col.shape[0] != val.shape[0] or rowptr.dim() != 1:
            raise ValueError("kg: col and val must have nnz entries, rowptr m + 1")
        m, nnz = int(rowptr.shape[0]) - 1, int(col.shape[0])
        super().__init__([m, n, nnz], [rowptr, col, val], val.dtype, **kw)
        self.m, self.n, self.nnz = m, int(n), nnz

    @property
    def nx(self):
        return self.n

    @property
    def ndata(self):
        return self.nnz


class TetEnergy(Problem):
    """f(u) = sum_e log1p(|G_e u_e|^2); conn int32 [N_e, 4], G [N_e, 12]."""
    kind = L.KG_TETENERGY

    def __init__(self, conn: torch.Tensor, G: torch.Tensor, nv: int, **kw):
        conn = _dev_tensor(conn, torch.int32)
        G = _dev_tensor(G)
        if conn.shape[-1] != 4 or G.shape[-1] != 12 or conn.shape[0] != G.shape[0]:
            raise ValueError("kg: conn must be [N_e, 4] and G [N_e, 12]")
        super().__init__([conn.shape[0], nv], [conn, G], G.dtype, **kw)
        self.ne, self.nv = int(conn.shape[0]), int(nv)

    @property
    def nx(self):
        return self.nv


class Laplace1D(Problem):
    """The paper's example f(x, b) = ||A (3x) - b||^2, A = tridiag(-1, 2, -1)."""
    kind = L.KG_LAPLACE1D

    def __init__(self, b: torch.Tensor, **kw):
        b = _dev_tensor(b)
        super().__init__([b.shape[0]], [b], b.dtype, **kw)
        self.n = int(b.shape[0])

    @property
    def nx(self):
        return self.n

    @property
    def ndata(self):
        return self.n


class BatchBuffers:
    """The x, f and gx buffers of one batch call with their device-pointer tables
    (Batch.bind).  Holds the tensors, so the addresses stay valid."""

    def __init__(self, xs, fs, gxs):
        self.xs, self.fs, self.gxs = list(xs), list(fs), list(gxs)
        self.tables = (L._table(self.xs), L._table(self.fs), L._table(self.gxs))


class Batch:
    """Many problems differentiated by one persistent launch (graph-replayed)."""

    def __init__(self, problems, arith="auto", strategy="auto", budget_bytes=0, stream=None):
        """budget_bytes: cap on the float-pair copies of dense A that the batch makes
        (kg_options.tape_budget_bytes; 0 = 1 GiB)."""
        self.problems = list(problems)
        opt = L.options(dtype=_DT[self.problems[0].dtype], arith=ARITHS[arith],
                        strategy=STRATEGIES[strategy], tape_budget_bytes=int(budget_bytes))
        self.handle = L.kg_batch_create([p.handle for p in self.problems], opt, stream)

    @property
    def config(self):
        """(arith, work items, persistent grid)."""
        return L.kg_batch_get_config(self.handle)

    def _check(self, xs, fs, gxs):
        # Lengths only: a batch call passes thousands of tensors, and checking each
        # would cost more host time than the batch takes on the GPU.  Entry i must be
        # laid out as for problems[i].grad (device, dtype, contiguous, nx elements;
        # fs[i] one element or None); check_buffers() checks that once.
        k = len(self.problems)
        if len(xs) != k or len(fs) != k or len(gxs) != k:
            raise ValueError(f"kg: the batch has {k} problems; xs, fs and gxs need one entry each")

    def check_buffers(self, xs, fs, gxs):
        """Full check of every entry of a set of batch buffers (call it once per set)."""
        self._check(xs, fs, gxs)
        for i, p in enumerate(self.problems):
            p._vec(xs[i], f"xs[{i}]")
            p._vec(gxs[i], f"gxs[{i}]")
            p._one(fs[i], f"fs[{i}]")

    def bind(self, xs, fs, gxs):
        """One set of buffers, checked in full and with its pointer tables built once.
        Building the tables costs about a microsecond a tensor of host time: for a batch
        of thousands of instances, milliseconds a call, as long as the batch's kernel.
        Pass the result to grad() / grad_loop() in place of (xs, fs, gxs)."""
        self.check_buffers(xs, fs, gxs)
        return BatchBuffers(xs, fs, gxs)

    def _tables(self, xs, fs, gxs):
        if isinstance(xs, BatchBuffers):
            if fs is not None or gxs is not None:
                raise ValueError("kg: pass either a BatchBuffers or (xs, fs, gxs)")
            if len(xs.xs) != len(self.problems):
                raise ValueError(f"kg: the batch has {len(self.problems)} problems; the bound "
                                 f"buffers {len(xs.xs)}")
            return xs.tables
        self._check(xs, fs, gxs)
        return L._table(xs), L._table(fs), L._table(gxs)

    def grad(self, xs, fs=None, gxs=None, stream=None):
        L.kg_grad_batched(self.handle, *self._tables(xs, fs, gxs), stream)

    def grad_loop(self, xs, fs=None, gxs=None, stream=None):
        L.kg_grad_batched_loop(self.handle, *self._tables(xs, fs, gxs), stream)

    def sync(self):
        L.kg_batch_sync(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            L.kg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

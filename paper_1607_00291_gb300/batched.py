"""Batches of contractions: one persistent launch over many problems.

``Plan`` wraps tc_plan_create / tc_plan_execute / tc_plan_destroy: the plan is
built once (validation, layouts, tile and split choice -- timed by the
autotuner when the environment has TC_AUTOTUNE=1 or names a cache file in
TC_AUTOTUNE_CACHE -- and a device copy of every descriptor), and ``execute`` only launches kernels on the current stream, so it
can be captured in a CUDA graph.  ``contract_batched`` is the one-shot form.
"""
import torch

from . import _lib as L


def _problem(A, labA, B, labB, C, labC, alpha=1.0, beta=0.0):
    for t in (A, B, C):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("A, B and C must be CUDA tensors")
    if not (A.dtype == B.dtype == C.dtype):
        raise TypeError("A, B and C must share one dtype")
    return (A, labA, B, labB, C, labC, float(alpha), float(beta))


class Plan:
    """A planned batch.  ``problems``: iterables (A, labA, B, labB, C, labC[,
    alpha[, beta]]) of CUDA tensors sharing one dtype and device; ``mode`` as
    in ``contract``.  The tensors must stay alive (and keep their storage)
    for as long as the plan is executed."""

    def __init__(self, problems, mode: str = "f64"):
        from . import _dtype_code, _mode_code
        probs = [_problem(*p) for p in problems]
        if not probs:
            raise ValueError("empty batch")
        self.device = probs[0][4].device
        self.dtype = _dtype_code(probs[0][4])
        self.mode = _mode_code(mode)
        self._keep = [probs]
        arr = (L.TcProblem * len(probs))()
        for i, (A, la, B, lb, C, lc, al, be) in enumerate(probs):
            if C.device != self.device or _dtype_code(C) != self.dtype:
                raise ValueError("all problems of a batch share one device and dtype")
            arr[i].alpha, arr[i].beta = al, be
            arr[i].A = L.make_tensor(tuple(A.shape), A.stride(), la, A.data_ptr(), self._keep)
            arr[i].B = L.make_tensor(tuple(B.shape), B.stride(), lb, B.data_ptr(), self._keep)
            arr[i].C = L.make_tensor(tuple(C.shape), C.stride(), lc, C.data_ptr(), self._keep)
        self._keep.append(arr)
        self._plan = L.c_vp(0)
        with torch.cuda.device(self.device):
            L.check(L.lib().tc_plan_create(self.dtype, self.mode, len(probs), arr, self._plan),
                    "tc_plan_create")
        self.count = len(probs)

    def execute(self, stream=None):
        if not self._plan:
            raise RuntimeError("plan destroyed")
        with torch.cuda.device(self.device):
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            L.check(L.lib().tc_plan_execute(self._plan, None, 0, L.c_vp(s.cuda_stream)),
                    "tc_plan_execute")

    def config(self, index: int) -> dict:
        """What the plan chose for problem `index`: tile rows and columns, the
        number of k-splits, and the batch's balance divisor (tc_plan_config)."""
        out = (L.c_i32 * 4)()
        L.check(L.lib().tc_plan_config(self._plan, int(index), out), "tc_plan_config")
        return {"bm": out[0], "bn": out[1], "splits": out[2], "balance": out[3]}

    @property
    def form(self) -> str:
        """The mainloop form of a tensor-core plan: "packed" or "gather"
        (tc_plan_form); "f64" for an FP64 plan."""
        if self.mode == L.TC_MODE_F64:
            return "f64"
        f = L.c_i32(0)
        L.check(L.lib().tc_plan_form(self._plan, f), "tc_plan_form")
        return {0: "gather", 3: "packed"}[f.value]

    def close(self):
        if getattr(self, "_plan", None):
            L.lib().tc_plan_destroy(self._plan)
            self._plan = L.c_vp(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def contract_batched(problems, mode: str = "f64"):
    """Run every problem (see ``Plan``) in one persistent launch; returns the
    list of C tensors."""
    p = Plan(problems, mode)
    try:
        p.execute()
        torch.cuda.current_stream(p.device).synchronize()
    finally:
        p.close()
    return [q[4] for q in p._keep[0]]

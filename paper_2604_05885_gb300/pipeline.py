"""Steps over point sets held in host memory, with transfers overlapped.

``HostPipeline`` runs build + kNN(k) + FoF(b) on a stream of equally sized
point sets that live in (pinned) host memory and returns the results to host
memory.  Device inputs and outputs are double buffered: while step i computes,
the upload of step i+1 and the download of step i-1 run on their own streams.
Events order every buffer reuse: an upload waits until the compute that read
its buffer two steps earlier has finished, a compute waits for its upload and
for the download of the outputs it overwrites, and a download waits for its
compute.  The work per step is exactly one jzt_build + jzt_tree_knn +
jzt_tree_fof, so results equal those of the one-call path.
"""
from __future__ import annotations

import torch

from . import Tree, alloc_workspace


class HostPipeline:
    def __init__(self, n: int, k: int, b: float, periodic_L: float = 0.0, params=None, device=None,
                 depth: int = 2):
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n, self.k, self.b, self.L, self.params = int(n), int(k), float(b), float(periodic_L), params
        self.depth = max(1, int(depth))
        self.ws = alloc_workspace(self.n, self.k, params, self.dev)
        self.x = [torch.empty((self.n, 3), dtype=torch.float32, device=self.dev) for _ in range(self.depth)]
        self.idx = [torch.empty((self.n, self.k), dtype=torch.int32, device=self.dev) for _ in range(self.depth)]
        self.d2 = [torch.empty((self.n, self.k), dtype=torch.float32, device=self.dev) for _ in range(self.depth)]
        self.lab = [torch.empty(self.n, dtype=torch.int32, device=self.dev) for _ in range(self.depth)]
        self.s_up = torch.cuda.Stream(device=self.dev)
        self.s_comp = torch.cuda.Stream(device=self.dev)
        self.s_down = torch.cuda.Stream(device=self.dev)
        self.ev_up = [None] * self.depth      # upload of slot done
        self.ev_comp = [None] * self.depth    # compute of slot done
        self.ev_down = [None] * self.depth    # download of slot done
        self.step_no = 0
        self.tree = None

    def submit(self, x_host: torch.Tensor, idx_host: torch.Tensor, d2_host: torch.Tensor, lab_host: torch.Tensor):
        """Enqueues one step: upload x_host, compute, download into the host outputs
        (all pinned CPU tensors of the step's shapes).  Returns at once."""
        s = self.step_no % self.depth
        self.step_no += 1
        with torch.cuda.stream(self.s_up):
            if self.ev_comp[s] is not None:
                self.s_up.wait_event(self.ev_comp[s])  # the compute that read this input slot
            self.x[s].copy_(x_host, non_blocking=True)
            self.ev_up[s] = torch.cuda.Event()
            self.ev_up[s].record(self.s_up)
        with torch.cuda.stream(self.s_comp):
            self.s_comp.wait_event(self.ev_up[s])
            if self.ev_down[s] is not None:
                self.s_comp.wait_event(self.ev_down[s])  # outputs of this slot have been read back
            self.tree = Tree(self.x[s], self.L, self.params, self.ws, stream=self.s_comp)
            self.tree.knn(self.k, out=(self.idx[s], self.d2[s]), stream=self.s_comp)
            self.tree.fof(self.b, out=self.lab[s], stream=self.s_comp)
            self.ev_comp[s] = torch.cuda.Event()
            self.ev_comp[s].record(self.s_comp)
        with torch.cuda.stream(self.s_down):
            self.s_down.wait_event(self.ev_comp[s])
            idx_host.copy_(self.idx[s], non_blocking=True)
            d2_host.copy_(self.d2[s], non_blocking=True)
            lab_host.copy_(self.lab[s], non_blocking=True)
            self.ev_down[s] = torch.cuda.Event()
            self.ev_down[s].record(self.s_down)

    def synchronize(self):
        for st in (self.s_up, self.s_comp, self.s_down):
            st.synchronize()

    def status(self, raise_on_error: bool = True) -> dict:
        self.synchronize()
        return self.tree.status(stream=self.s_comp, raise_on_error=raise_on_error)

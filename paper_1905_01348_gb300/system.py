"""A PT-CN system whose workspace and stream come from PyTorch (device memory plumbing only)."""
from __future__ import annotations

import numpy as np

from . import _native as nat


class System:
    """Owns one pt_system handle and the device workspace it runs in.

    params: workload dictionary (see synthetic.si_workload); psi0: (n_orb, npw)
    complex128 start coefficients, or None for the library's seeded ones
    (pt_seeded_coefficients of params["seed"]). The workspace is a torch uint8
    tensor on ``device`` (allocated here, or passed in as ``workspace``: at least
    pt_workspace_size bytes, 256-byte aligned, owned by the caller); all work is
    enqueued on ``stream``, else torch's current stream of that device.
    """

    def __init__(self, params: dict, psi0, device: str = "cuda:0", stream=None, workspace=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.params = nat.make_params(params)
        self.npw = nat.pt_basis_size(self.params)
        self.n_orb = self.params.n_orb
        self.ws_bytes = nat.pt_workspace_size(self.params)
        if workspace is None:
            workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        elif workspace.numel() < self.ws_bytes or workspace.dtype != torch.uint8:
            raise ValueError("workspace: a uint8 device tensor of at least pt_workspace_size bytes is required")
        self.workspace = workspace
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.handle = nat.pt_init_system(self.params, psi0, self.workspace.data_ptr(), self.ws_bytes,
                                         self.stream.cuda_stream)

    # -- state -------------------------------------------------------------
    def orbitals(self) -> np.ndarray:
        return nat.pt_get_orbitals(self.handle, self.n_orb, self.npw)

    def set_orbitals(self, psi: np.ndarray) -> None:
        nat.pt_set_orbitals(self.handle, psi)

    def get_state(self):
        """(Psi, W = V_X Psi, step index) with Psi, W as (n_orb, npw) complex128 host arrays."""
        psi = np.empty((self.n_orb, self.npw), dtype=np.complex128)
        w = np.empty_like(psi)
        step = nat.pt_get_state(self.handle, psi, w)
        return psi, w, step

    def set_state(self, psi: np.ndarray, w: np.ndarray, step: int) -> None:
        nat.pt_set_state(self.handle, psi, w, step)

    def observables(self):
        return nat.pt_observables(self.handle)

    def orbitals_device(self):
        """A torch view (n_orb, npw) complex128 of the current device orbitals."""
        ptr = nat.pt_orbitals_device(self.handle)
        base = self.workspace.data_ptr()
        off = ptr - base
        nbytes = self.n_orb * self.npw * 16
        return self.workspace[off:off + nbytes].view(self.torch.complex128).view(self.n_orb, self.npw)

    # -- operations ------------------------------------------------------------
    def exchange(self):
        """V_X Psi of the current orbitals as a (n_orb, npw) complex128 device tensor."""
        out = self.torch.empty((self.n_orb, self.npw), dtype=self.torch.complex128, device=self.device)
        nat.pt_exchange(self.handle, out.data_ptr())
        return out

    def apply_h(self, X, fock_mode: int = nat.PT_FOCK_EXACT):
        """H X for a (m, npw) complex128 device tensor X (m <= n_orb)."""
        X = X.contiguous()
        Y = self.torch.empty_like(X)
        nat.pt_apply_h(self.handle, X.data_ptr(), Y.data_ptr(), X.shape[0], fock_mode)
        return Y

    def build_ace(self) -> None:
        nat.pt_build_ace(self.handle)

    def step(self):
        return nat.pt_cn_step(self.handle)

    def rk4_step(self):
        """One explicit RK4 step (the comparison integrator); returns the step info dict."""
        return nat.pt_rk4_step(self.handle)

    def propagate(self, nsteps: int):
        return nat.pt_propagate(self.handle, nsteps)

    def close(self) -> None:
        """Destroy the handle and release the workspace (its memory returns to the allocator
        now, even while other objects still refer to this System)."""
        if getattr(self, "handle", None) is not None:
            nat.pt_destroy(self.handle)
            self.handle = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several systems stepped together (pt_batch_*): their pair tiles share launch groups.

    systems: System objects with the same grid, precision, cell, cutoff and kernel; each
    keeps its own stream. The batch workspace and the stream of the merged pair kernels
    come from PyTorch. pair_tile / tiles_per_launch: the tile edge and launch-group size
    (0: automatic; the autotuner's table gives tuned values). priority: CUDA priority of
    the batch's stream (0 normal, negative higher). workspace: optional caller-owned uint8
    device tensor of at least the batch workspace size (else one is allocated).
    """

    @staticmethod
    def workspace_size(systems, pair_tile: int = 0, tiles_per_launch: int = 0) -> int:
        return max(256, nat.pt_batch_workspace_size([s.handle for s in systems], pair_tile, tiles_per_launch))

    def __init__(self, systems, pair_tile: int = 0, tiles_per_launch: int = 0, priority: int = 0, workspace=None):
        import torch
        self.torch = torch
        self.systems = list(systems)
        dev = self.systems[0].device
        handles = [s.handle for s in self.systems]
        self.ws_bytes = nat.pt_batch_workspace_size(handles, pair_tile, tiles_per_launch)
        if workspace is None:
            workspace = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        elif workspace.numel() < max(self.ws_bytes, 256) or workspace.dtype != torch.uint8:
            raise ValueError("workspace: a uint8 device tensor of at least the batch workspace size is required")
        self.workspace = workspace
        self.stream = torch.cuda.Stream(dev, priority=priority)
        self.handle = nat.pt_batch_create(handles, pair_tile, tiles_per_launch, self.workspace.data_ptr(),
                                          self.ws_bytes, self.stream.cuda_stream)

    def step(self):
        """One PT-CN step of every system: (status, [step info per system])."""
        return nat.pt_batch_step(self.handle, len(self.systems))

    def exchange(self):
        """V_X Psi of every system's current orbitals, one (n_orb, npw) complex128 device tensor each."""
        outs = [self.torch.empty((s.n_orb, s.npw), dtype=self.torch.complex128, device=s.device) for s in self.systems]
        nat.pt_batch_exchange(self.handle, [o.data_ptr() for o in outs])
        return outs

    def close(self) -> None:
        if getattr(self, "handle", None) is not None:
            nat.pt_batch_destroy(self.handle)
            self.handle = None
        self.workspace = None
        self.systems = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Shared helpers of the GPU tests: a libqsa state over a torch buffer and the
floating-point parity check against the oracle."""
import numpy as np

import oracle

FID_TOL = 1e-5   # 1 - |<psi_gpu|psi_ref>|^2
AMP_TOL = 1e-5   # max |psi_gpu - psi_ref|


class GState:
    """A libqsa state over a torch-owned complex64 buffer on cuda:0."""

    def __init__(self, q, torch, n, init=None):
        self.q, self.torch, self.n = q, torch, n
        self.buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda:0")
        if init is not None:
            self.buf.copy_(torch.from_numpy(np.ascontiguousarray(init, dtype=np.complex64)))
            torch.cuda.synchronize()
        self.stream = torch.cuda.current_stream().cuda_stream
        self.h = q.qsa_state_create_ex(n, self.buf.data_ptr(), self.buf.numel() * 8, self.stream,
                                       0 if init is not None else 1)

    def stored(self):
        self.q.qsa_state_sync(self.h)
        return self.buf.cpu().numpy().astype(np.complex128)

    def logical(self):
        return oracle.decode_state(self.stored(), self.q.qsa_get_layout(self.h))

    def close(self):
        self.q.qsa_state_destroy(self.h)


def check_close(ref, got, fid_tol=FID_TOL, amp_tol=AMP_TOL):
    """1 - F within fid_tol on both sides (F is not renormalised, so a norm
    that grew counts like one that shrank) and the largest amplitude
    difference within amp_tol."""
    f = oracle.fidelity(ref, got)
    e = oracle.max_abs_diff(ref, got)
    assert abs(1 - f) <= fid_tol and e <= amp_tol, (1 - f, e)
    return 1 - f, e

"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module only *generates inputs*: gate matrices, target tuples, random
graphs, Pauli branch choices.  It holds none of the simulation arithmetic (no
state update, no fusion, no sampling) and imports neither the oracle nor the
CUDA library.

Every random choice is drawn from ``numpy.random.default_rng`` seeded by the
caller, so the CUDA path and the oracle always see identical inputs.  The
circuit families stand in for the paper's missing OpenQASM inputs
(``rand{N}x{d}``, ``qft{N}``, the QAOA application circuits, §V-A
"Workloads"); their shapes follow the paper's description where it gives one.

Matrix convention (§II): a gate on the ordered tuple (q_0..q_{k-1}) is a
2^k x 2^k complex matrix whose row / column bit j belongs to q_j.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np


@dataclass
class Op:
    targets: Tuple[int, ...]
    matrix: np.ndarray            # complex128, 2^k x 2^k
    diag: bool = False            # eligible for the diagonal marker (§IV-C)
    name: str = ""

    @property
    def k(self) -> int:
        return len(self.targets)


# ---------------------------------------------------------------------------
# Gate matrices
# ---------------------------------------------------------------------------
S2 = 1.0 / np.sqrt(2.0)
H = np.array([[S2, S2], [S2, -S2]], dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
# CNOT on the tuple (control, target): index = control + 2*target.
CNOT = np.zeros((4, 4), dtype=np.complex128)
for _c in range(4):
    _ctl, _tgt = _c & 1, (_c >> 1) & 1
    _r = _ctl | ((_tgt ^ _ctl) << 1)
    CNOT[_r, _c] = 1.0
SWAP = np.zeros((4, 4), dtype=np.complex128)
for _c in range(4):
    SWAP[((_c & 1) << 1) | (_c >> 1), _c] = 1.0
PAULIS = [I2, X, Y, Z]


def cphase(phi: float) -> np.ndarray:
    return np.diag([1, 1, 1, np.exp(1j * phi)]).astype(np.complex128)


def rx(beta: float) -> np.ndarray:
    """RX(beta) = exp(-i beta X / 2)."""
    c, s = np.cos(beta / 2), np.sin(beta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def zz(gamma: float) -> np.ndarray:
    """ZZ(gamma) = exp(-i gamma Z(x)Z / 2)."""
    a, b = np.exp(-0.5j * gamma), np.exp(0.5j * gamma)
    return np.diag([a, b, b, a]).astype(np.complex128)


def haar_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(d): QR of a complex Ginibre matrix with the phases of
    diag(R) divided out (Mezzadri, Notices AMS 2007)."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def inverse(ops: Sequence[Op]) -> List[Op]:
    """The inverse circuit: conjugate transposes in reverse order."""
    return [Op(o.targets, o.matrix.conj().T.copy(), o.diag, o.name + "^-1") for o in reversed(ops)]


# ---------------------------------------------------------------------------
# Circuit families
# ---------------------------------------------------------------------------

def brick_layers(n: int, layers: int, rng: np.random.Generator, first_layer: int = 0) -> List[Op]:
    """Each layer: Haar U(2) on every qubit, then CZ on alternating
    neighbour pairs — even layers (0,1),(2,3),..., odd layers (1,2),(3,4),...
    on an open chain."""
    ops: List[Op] = []
    for l in range(first_layer, first_layer + layers):
        for q in range(n):
            ops.append(Op((q,), haar_unitary(2, rng), False, "u2"))
        for a in range(l % 2, n - 1, 2):
            ops.append(Op((a, a + 1), CZ.copy(), True, "cz"))
    return ops


def brick_circuit(n: int = 12, layers: int = 20, seed: int = 0) -> List[Op]:
    """Plain per-gate workload: 20 brick layers at N=12 from |0...0>."""
    return brick_layers(n, layers, np.random.default_rng(seed))


def qft_ops(n: int) -> List[Op]:
    """QFT|x> = 2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y>, qubit 0 least
    significant: for j = n-1 .. 0, H on j then controlled phases
    CP(pi / 2^(j-m)) on (m, j) for m = j-1 .. 0; then reverse the bit order
    with SWAPs."""
    ops: List[Op] = []
    for j in range(n - 1, -1, -1):
        ops.append(Op((j,), H.copy(), False, "h"))
        for m in range(j - 1, -1, -1):
            ops.append(Op((m, j), cphase(np.pi / (1 << (j - m))), True, "cp"))
    for a in range(n // 2):
        ops.append(Op((a, n - 1 - a), SWAP.copy(), False, "swap"))
    return ops


def basis_prep(n: int, x: int) -> List[Op]:
    return [Op((q,), X.copy(), False, "x") for q in range(n) if (x >> q) & 1]


def random_matching(n: int, rng: np.random.Generator) -> List[Tuple[int, int]]:
    """Fisher-Yates shuffle of 0..n-1, then consecutive entries paired."""
    perm = rng.permutation(n)
    return [(int(perm[2 * i]), int(perm[2 * i + 1])) for i in range(n // 2)]


def fusion_circuit(n: int = 28, layers: int = 40, seed: int = 0, with_inverse: bool = True):
    """QFT on a seeded random basis state, then ``layers`` layers of Haar U(2)
    on every qubit plus Haar U(4) on a random perfect matching, then (when
    ``with_inverse``) the inverse of everything, returning to |0...0>.
    Returns (ops, x0)."""
    rng = np.random.default_rng(seed)
    x0 = int(rng.integers(0, 1 << n))
    fwd = basis_prep(n, x0) + qft_ops(n)
    for _ in range(layers):
        for q in range(n):
            fwd.append(Op((q,), haar_unitary(2, rng), False, "u2"))
        for a, b in random_matching(n, rng):
            fwd.append(Op((a, b), haar_unitary(4, rng), False, "u4"))
    ops = fwd + (inverse(fwd) if with_inverse else [])
    return ops, x0


def wide_circuit(n: int, n_ops: int = 200, widths: Sequence[int] = (5, 6), seed: int = 0) -> List[Op]:
    """``n_ops`` Haar-random U(2^k) with k cycling through ``widths``, target
    sets uniform without replacement over 0..n-1 (mixed low / high bits), in
    random order."""
    rng = np.random.default_rng(seed)
    ops = []
    for i in range(n_ops):
        k = int(widths[i % len(widths)])
        t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        ops.append(Op(t, haar_unitary(1 << k, rng), False, f"u{1 << k}"))
    return ops


def random_3regular(n: int, rng: np.random.Generator, max_tries: int = 10000) -> List[Tuple[int, int]]:
    """Random 3-regular simple graph by the pairing (configuration) model,
    rejecting self-loops and multi-edges.  n must be even."""
    assert n % 2 == 0
    for _ in range(max_tries):
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for a, b in pairs:
            a, b = int(a), int(b)
            if a == b or (min(a, b), max(a, b)) in edges:
                ok = False
                break
            edges.add((min(a, b), max(a, b)))
        if ok:
            return sorted(edges)
    raise RuntimeError("no simple 3-regular graph found")


def qaoa_circuit(n: int = 30, p: int = 8, seed: int = 0):
    """QAOA on a random 3-regular graph: H on every qubit, then p rounds of
    ZZ(gamma_l) on every edge and RX(beta_l) on every qubit; angles uniform in
    [0, 2 pi).  Returns (ops, edges)."""
    rng = np.random.default_rng(seed)
    edges = random_3regular(n, rng)
    gam = rng.uniform(0, 2 * np.pi, size=p)
    bet = rng.uniform(0, 2 * np.pi, size=p)
    ops = [Op((q,), H.copy(), False, "h") for q in range(n)]
    for l in range(p):
        for a, b in edges:
            ops.append(Op((a, b), zz(gam[l]), True, "zz"))
        for q in range(n):
            ops.append(Op((q,), rx(bet[l]), False, "rx"))
    return ops, edges


def ghz_ops(n: int) -> List[Op]:
    """H on qubit 0, then CNOT(0 -> q) for q = 1..n-1."""
    return [Op((0,), H.copy(), False, "h")] + [Op((0, q), CNOT.copy(), False, "cx") for q in range(1, n)]


def random_clifford(n: int, n_gates: int, seed: int = 0) -> List[Op]:
    """Random gates from {H, S, CNOT, CZ} on random qubits."""
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(n_gates):
        g = int(rng.integers(0, 4))
        if g == 0:
            ops.append(Op((int(rng.integers(0, n)),), H.copy(), False, "h"))
        elif g == 1:
            ops.append(Op((int(rng.integers(0, n)),), S.copy(), True, "s"))
        else:
            a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
            ops.append(Op((a, b), (CNOT if g == 2 else CZ).copy(), g == 3, "cx" if g == 2 else "cz"))
    return ops


def trajectory_circuit(n: int, depth: int, rng: np.random.Generator, p: float = 1e-3) -> Tuple[List[Op], int]:
    """One noisy trajectory: ``depth`` brick layers of U(2) + CZ.  After each
    gate, with probability p, a Pauli branch is inserted: one of X, Y, Z
    (p/3 each) after a one-qubit gate, one of the 15 non-identity two-qubit
    Pauli strings (p/15 each) after a CZ (depolarising channel, uniform over
    non-identity strings, §IV-A).  Returns (ops, number of inserted Paulis)."""
    base = brick_layers(n, depth, rng)
    ops: List[Op] = []
    n_ins = 0
    for op in base:
        ops.append(op)
        if rng.random() < p:
            n_ins += 1
            if op.k == 1:
                P = PAULIS[1 + int(rng.integers(0, 3))]
                ops.append(Op(op.targets, P.copy(), False, "pauli"))
            else:
                s = 1 + int(rng.integers(0, 15))
                P = np.kron(PAULIS[s >> 2], PAULIS[s & 3])  # bit 0 <-> targets[0]
                ops.append(Op(op.targets, P.astype(np.complex128), False, "pauli2"))
    return ops, n_ins


def trajectory_batch(n_traj: int = 256, n: int = 20, dmin: int = 10, dmax: int = 60, seed: int = 0,
                     p: float = 1e-3):
    """``n_traj`` trajectories with depths uniform in [dmin, dmax]; trajectory
    t uses the generator seeded by (seed, t).  Returns (list of op lists,
    depths)."""
    trajs, depths = [], []
    for t in range(n_traj):
        rng = np.random.default_rng([seed, t])
        d = int(rng.integers(dmin, dmax + 1))
        ops, _ = trajectory_circuit(n, d, rng, p)
        trajs.append(ops)
        depths.append(d)
    return trajs, depths


# ---------------------------------------------------------------------------
# Channels (Kraus lists) for the density-matrix path
# ---------------------------------------------------------------------------
@dataclass
class Channel:
    targets: Tuple[int, ...]
    kraus: List[np.ndarray]       # each complex128, 2^k x 2^k, bit j <-> targets[j]
    name: str = ""


def pauli_string(s: int, k: int) -> np.ndarray:
    """Tensor product of PAULIS[(s >> 2j) & 3] with factor j on tuple bit j."""
    m = np.ones((1, 1), dtype=np.complex128)
    for j in range(k):
        m = np.kron(PAULIS[(s >> (2 * j)) & 3], m)
    return m


def depolarising_kraus(k: int, p: float) -> List[np.ndarray]:
    """k-qubit depolarising noise, uniform over the 4^k - 1 non-identity Pauli
    strings: sqrt(1-p) I and sqrt(p / (4^k - 1)) P."""
    w = np.sqrt(p / (4 ** k - 1))
    return [np.sqrt(1 - p) * np.eye(1 << k, dtype=np.complex128)] + [w * pauli_string(s, k)
                                                                     for s in range(1, 4 ** k)]


def amplitude_damping_kraus(gamma: float) -> List[np.ndarray]:
    return [np.array([[1, 0], [0, np.sqrt(1 - gamma)]], dtype=np.complex128),
            np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)]


def random_kraus(k: int, r: int, rng: np.random.Generator) -> List[np.ndarray]:
    """r Kraus operators of a random trace-preserving map: the 2^k-row blocks
    of a random (r 2^k) x 2^k isometry (QR of a complex Gaussian matrix)."""
    d = 1 << k
    z = rng.standard_normal((r * d, d)) + 1j * rng.standard_normal((r * d, d))
    qm, _ = np.linalg.qr(z)
    return [np.ascontiguousarray(qm[i * d:(i + 1) * d, :]) for i in range(r)]


def noisy_ghz_channels(n: int, p: float = 1e-2) -> List[Channel]:
    """GHZ preparation with depolarising noise p after the H and after each
    CNOT (two-qubit depolarising on the CNOT's pair), the noisy-GHZ shape of
    §V (routing benchmark); every gate is a one-operator channel."""
    out: List[Channel] = []
    for op in ghz_ops(n):
        out.append(Channel(op.targets, [op.matrix], op.name))
        out.append(Channel(op.targets, depolarising_kraus(op.k, p), f"dep{op.k}"))
    return out


def random_channel_circuit(n: int, n_ch: int, rng: np.random.Generator, kmax: int = 3) -> List[Channel]:
    """A mix of Haar unitaries (one Kraus operator) and random channels of
    1..kmax qubits with 1..4 Kraus operators on random target tuples."""
    out: List[Channel] = []
    for _ in range(n_ch):
        k = int(rng.integers(1, kmax + 1))
        t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        if rng.random() < 0.5:
            out.append(Channel(t, [haar_unitary(1 << k, rng)], "u"))
        else:
            out.append(Channel(t, random_kraus(k, int(rng.integers(1, 5)), rng), "kraus"))
    return out


def random_state(n: int, seed: int = 0, zero_frac: float = 0.0) -> np.ndarray:
    """A normalised complex128 random state; a fraction of entries can be set
    exactly to zero (for sampler edge cases)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    if zero_frac > 0:
        v[rng.random(1 << n) < zero_frac] = 0
    return v / np.linalg.norm(v)

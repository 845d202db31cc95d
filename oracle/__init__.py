"""FP64 CPU oracle — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this package.  It shares no code with the CUDA
library (``paper_2608_16940_gb300``) and never imports it.

Contents
--------
* ``qsa_oracle.c`` (built into ``liboracle.so`` by :func:`build`): the plain
  single-threaded FP64 state-vector update, probabilities, <Z>, Philox4x64-10
  and the fixed-point CDF sampler.
* this module: ctypes wrappers plus plain numpy restatements of
  - the diagonal branch of Alg. 2 (elementwise multiply by the entry the
    target bits index) and the fused diagonal of a block of diagonal gates,
  - the product lowering of a block of one-qubit factors on distinct qubits
    and the grouping of a circuit into product units,
  - layer blocks (one-qubit factors preceded by one- and two-qubit diagonal
    gates on any qubits, one tile pass) and the commutation-aware grouping of
    a circuit into them; the prefix of a circuit that a plan for |0...0>
    prepares as a product state times diagonal gates, and that state,
  - density-matrix evolution by Kraus operators, its column-major
    vectorisation and the superoperator of a channel,
  - the Kronecker embedding and block product used by fusion (§IV-C: "within a
    block, matrices remain in circuit order, with later gates multiplied on
    the left"),
  - the fusion partition dynamic program (§IV-C, Eq. dp-recurrence) and the
    plain width-limit greedy partition,
  - the replay of on-demand promotions under first-free and farthest-next-use
    victim choice (§IV-D, Corollary "ideal minimal demand-promotion count"),
  - the cost-model network (37 -> 64 -> 64 -> 1, ReLU, MSE on log-seconds)
    forward, backward and one Adam step (Kingma & Ba 2015, Algorithm 1),
  - fidelity metrics.

Pins for every function live in ``tests/test_oracle_*.py``.  Functions with no
pin beyond their definition say so in their docstring ("parity unpinned").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc.  ``-ffp-contract=off`` keeps every
    product and sum rounded separately (no fused multiply-add), which the
    sampler's fixed-point weights rely on."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               _SRC, "-o", _LIB_PATH]
        subprocess.check_call(cmd)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.orc_apply.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, dp]
        L.orc_apply.restype = ctypes.c_int
        L.orc_probabilities.argtypes = [dp, ctypes.c_int, dp]
        L.orc_probabilities.restype = None
        L.orc_expect_z.argtypes = [dp, ctypes.c_int, ctypes.c_uint64]
        L.orc_expect_z.restype = ctypes.c_double
        L.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.orc_philox4x64_10.restype = None
        L.orc_sample.argtypes = [dp, ctypes.c_int, ip, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                 ctypes.c_double, u64p, ctypes.POINTER(ctypes.c_uint8)]
        L.orc_sample.restype = ctypes.c_int
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# State-vector operations (C)
# ---------------------------------------------------------------------------

def zero_state(n: int) -> np.ndarray:
    """|0...0>: psi_0 = 1 (§II)."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply(psi: np.ndarray, targets: Sequence[int], mat: np.ndarray) -> None:
    """In place: apply the 2^k x 2^k matrix ``mat`` on the ordered tuple
    ``targets`` (little-endian, §II) of the canonical-order state ``psi``."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    n = int(psi.size).bit_length() - 1
    k = len(targets)
    m = np.ascontiguousarray(mat, dtype=np.complex128)
    assert m.shape == (1 << k, 1 << k)
    t = (ctypes.c_int * k)(*[int(q) for q in targets])
    rc = lib().orc_apply(_dptr(psi.view(np.float64)), n, t, k, _dptr(m.view(np.float64)))
    if rc != 0:
        raise ValueError("oracle apply: invalid arguments")


def diag_index(n: int, targets: Sequence[int]) -> np.ndarray:
    """c(x) for every canonical index x: bit j of c is bit targets[j] of x."""
    x = np.arange(1 << n, dtype=np.int64)
    c = np.zeros_like(x)
    for j, t in enumerate(targets):
        c |= ((x >> int(t)) & 1) << j
    return c


def apply_diag(psi: np.ndarray, targets: Sequence[int], d: np.ndarray) -> None:
    """In place: the diagonal branch of Alg. 2 (axis-shifted lowering), "multiply
    each amplitude by the diagonal entry indexed by the target bits":
    psi[x] <- d[c(x)], with bit j of c equal to bit targets[j] of x (§II
    little-endian order); the layout is unchanged."""
    n = int(psi.size).bit_length() - 1
    d = np.asarray(d, dtype=np.complex128)
    assert d.shape == (1 << len(targets),)
    psi *= d[diag_index(n, targets)]


def fuse_diag(gates: Sequence, block_targets: Sequence[int]) -> np.ndarray:
    """Diagonal of the fused block of diagonal gates on ``block_targets``
    (ascending union of the gates' targets): entry c is the product, in circuit
    order, of each gate's diagonal entry at the bits of c that are its targets
    (§IV-C block product restricted to the diagonal mode)."""
    u = len(block_targets)
    pos = {int(q): i for i, q in enumerate(block_targets)}
    d = np.ones(1 << u, dtype=np.complex128)
    cs = np.arange(1 << u, dtype=np.int64)
    for g in gates:
        gi = np.zeros_like(cs)
        for j, t in enumerate(g.targets):
            gi |= ((cs >> pos[int(t)]) & 1) << j
        d = np.diag(np.asarray(g.matrix, dtype=np.complex128))[gi] * d
    return d


def apply_product(psi: np.ndarray, targets: Sequence[int], factors: Sequence[np.ndarray]) -> None:
    """In place: the product operator U_{k-1} (x) ... (x) U_0 with the 2x2
    factor U_j on qubit targets[j] (distinct), i.e. each factor applied as its
    own one-qubit gate (they act on different qubits, so order is free).  A
    structured fused block (§IV-D: such blocks may use cheaper lowerings)."""
    assert len(set(int(t) for t in targets)) == len(targets)
    for t, u in zip(targets, factors):
        apply(psi, (int(t),), np.asarray(u, dtype=np.complex128))


def fuse_product(ops: Sequence) -> Tuple[List[int], List[np.ndarray]]:
    """Factors of a product unit: for each qubit (ascending), the product of
    its one-qubit ops in circuit order, later ops on the left (§IV-C)."""
    f = {}
    for o in ops:
        q = int(o.targets[0])
        f[q] = np.asarray(o.matrix, dtype=np.complex128) @ f.get(q, np.eye(2, dtype=np.complex128))
    t = sorted(f)
    return t, [f[q] for q in t]


def product_units(ops: Sequence, kmax_prod: int) -> List[Tuple[int, int]]:
    """Product units of a circuit: maximal runs of consecutive non-diagonal
    one-qubit ops touching at most ``kmax_prod`` distinct qubits (a run of
    width 1 is an ordinary op); every other op is a unit of its own.  Returns
    half-open op ranges in order."""
    units, i, n_ops = [], 0, len(ops)
    while i < n_ops:
        o = ops[i]
        if kmax_prod >= 2 and len(o.targets) == 1 and not o.diag:
            qs, j = {o.targets[0]}, i + 1
            while j < n_ops and len(ops[j].targets) == 1 and not ops[j].diag:
                if ops[j].targets[0] not in qs and len(qs) == kmax_prod:
                    break
                qs.add(ops[j].targets[0])
                j += 1
            units.append((i, j))
            i = j
        else:
            units.append((i, i + 1))
            i += 1
    return units


# ---------------------------------------------------------------------------
# Layer blocks: diagonal gates then a layer of one-qubit factors
# ---------------------------------------------------------------------------
LAYER_TILE_BITS = 12   # a tile of 2^12 amplitudes
LAYER_LOW_BITS = 3     # its lowest 3 bits are the state's lowest 3 positions


def layer_fits(positions: Iterable[int], n: int) -> bool:
    """The factor positions fit one tile: a tile of T = min(12, n) bits keeps
    the lowest min(3, T) positions, so at most T - min(3, T) factor positions
    may lie above them."""
    T = min(LAYER_TILE_BITS, n)
    low = min(LAYER_LOW_BITS, T)
    return sum(1 for p in positions if p >= low) <= T - low


def apply_layer(psi: np.ndarray, diag_ops: Sequence, targets: Sequence[int], factors: Sequence[np.ndarray]) -> None:
    """The layer block's definition (a structured fused block, §IV-D): every
    diagonal gate, then the one-qubit factor j on targets[j] (distinct
    qubits).  Applied gate by gate with ``apply``."""
    for g in diag_ops:
        apply(psi, g.targets, g.matrix)
    for t, f in zip(targets, factors):
        apply(psi, (t,), f)


def layer_units(ops: Sequence, n: int, layout: Sequence[int] | None = None, lookahead: int = 256):
    """Commutation-aware grouping into layer blocks.

    Ops are taken from the front of the pending stream.  A stream whose first
    op is neither one-qubit nor a diagonal gate on at most two qubits emits
    that op as a plain unit.  Otherwise a block is grown by scanning the
    pending ops in circuit order:

    * a diagonal gate on k <= 2 qubits joins the diagonal part when none of
      its qubits has a factor in the block yet and no skipped non-diagonal op
      touches them (it then moves ahead of the skipped ops, which it commutes
      with, and ahead of the block's factors, which act on other qubits);
    * a one-qubit op joins the factor of its qubit (later ops on the left) when
      no skipped op touches that qubit and the factor qubits' physical
      positions still fit a tile (``layer_fits``);
    * any other op is skipped and blocks its qubits: for everything, if it is
      not diagonal; for non-diagonal ops only, if it is diagonal.

    After more than ``lookahead`` skips the scan stops.  The block is the
    diagonal part then the factors (each in circuit order); skipped ops stay
    pending in order.  Returns (order, units): ``order`` lists the input op
    indices in execution order and each unit is (start, end, is_layer, n_diag)
    over ``order``, the first n_diag ops of a layer unit being its diagonal
    part."""
    L = list(range(n)) if layout is None else list(layout)
    pending = list(range(len(ops)))
    order: List[int] = []
    units = []
    while pending:
        first = ops[pending[0]]
        if not (len(first.targets) == 1 or (first.diag and len(first.targets) <= 2)):
            units.append((len(order), len(order) + 1, False, 0))
            order.append(pending.pop(0))
            continue
        diag_part, factor_part = [], []
        fq = set()
        blocked_nondiag, blocked_all = set(), set()
        skips = 0
        for idx in pending:
            op = ops[idx]
            Q = set(op.targets)
            if op.diag and len(Q) <= 2 and not (Q & fq) and not (Q & blocked_nondiag):
                diag_part.append(idx)
            elif len(Q) == 1 and not (Q & blocked_all) and layer_fits([L[q] for q in fq | Q], n):
                factor_part.append(idx)
                fq |= Q
            else:
                blocked_all |= Q
                if not op.diag:
                    blocked_nondiag |= Q
                skips += 1
                if skips > lookahead:
                    break
        taken = set(diag_part) | set(factor_part)
        start = len(order)
        order += diag_part + factor_part
        units.append((start, len(order), True, len(diag_part)))
        pending = [x for x in pending if x not in taken]
    return order, units


def zero_init_prefix(ops: Sequence) -> int:
    """Length of the prefix a plan for |0...0> prepares in one write-only pass:
    ops are taken in circuit order while each is a one-qubit op on a qubit no
    taken diagonal gate touches (it multiplies that qubit's state) or a
    diagonal gate on at most two qubits (it is applied after all of them).
    The prefix leaves psi(x) = prod_q a_q[x_q] * prod_g d_g(x), a_q the qubit's
    ops applied to |0>."""
    diag_touched = set()
    for i, op in enumerate(ops):
        t = tuple(op.targets)
        if len(t) == 1 and t[0] not in diag_touched:
            continue
        if op.diag and len(t) <= 2:
            diag_touched |= set(t)
            continue
        return i
    return len(ops)


def zero_init_state(n: int, ops: Sequence) -> np.ndarray:
    """The prefix's state from its closed form: per-qubit vectors a_q (the
    qubit's one-qubit ops applied to |0>), their Kronecker product, then the
    diagonal gates' entries (``apply_diag``)."""
    a = [np.array([1.0, 0.0], dtype=np.complex128) for _ in range(n)]
    diags = []
    for op in ops:
        if len(op.targets) == 1 and not diags_touch(diags, op.targets[0]):
            a[op.targets[0]] = np.asarray(op.matrix, dtype=np.complex128) @ a[op.targets[0]]
        else:
            diags.append(op)
    psi = np.ones(1, dtype=np.complex128)
    for q in range(n):
        psi = np.kron(a[q], psi)      # qubit q is bit q of the index
    for g in diags:
        apply_diag(psi, g.targets, np.diag(np.asarray(g.matrix, dtype=np.complex128)).copy())
    return psi


def diags_touch(diags, q: int) -> bool:
    return any(q in g.targets for g in diags)


def layer_block(ops: Sequence, idx: Sequence[int], n_diag: int):
    """Split one layer unit (op indices in execution order, the first n_diag
    of them diagonal gates) into its diagonal gates and its per-qubit factors
    (qubits ascending, each the product of its ops in order, later ops on the
    left)."""
    diag_ops = [ops[i] for i in idx[:n_diag]]
    fac = {}
    for i in idx[n_diag:]:
        q = ops[i].targets[0]
        fac[q] = np.asarray(ops[i].matrix, dtype=np.complex128) @ fac.get(q, np.eye(2, dtype=np.complex128))
    qs = sorted(fac)
    return diag_ops, qs, [fac[q] for q in qs]


def dm_zero(n: int) -> np.ndarray:
    """|0...0><0...0| as a 2^n x 2^n matrix."""
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[0, 0] = 1.0
    return rho


def dm_apply_channel(rho: np.ndarray, targets: Sequence[int], kraus: Sequence[np.ndarray]) -> np.ndarray:
    """rho' = sum_i E_i rho E_i^dagger with each Kraus operator E_i (2^k x 2^k)
    acting on ``targets`` (§IV-B density-matrix wrapper; a unitary is the
    single-operator channel).  Plain matrix products with the embedded
    operators (full_operator), small n only."""
    n = int(rho.shape[0]).bit_length() - 1
    out = np.zeros_like(rho)
    for E in kraus:
        M = full_operator(n, targets, np.asarray(E, dtype=np.complex128))
        out += M @ rho @ M.conj().T
    return out


def dm_vec(rho: np.ndarray) -> np.ndarray:
    """Column-major vectorisation: index row + 2^n * column (the lower n bits
    select the row, the upper n bits the column)."""
    return np.ascontiguousarray(rho.T).reshape(-1)


def dm_unvec(v: np.ndarray) -> np.ndarray:
    d = int(round(np.sqrt(v.size)))
    return v.reshape(d, d).T.copy()


def dm_superoperator(kraus: Sequence[np.ndarray]) -> np.ndarray:
    """sum_i conj(E_i) (x) E_i: the channel on the 2k axes of vec(rho), with the
    original factor on the lower (row) bits and the conjugate on the upper
    (column) bits."""
    return sum(np.kron(np.conj(E), E) for E in kraus)


def run_circuit(n: int, ops: Iterable, psi: np.ndarray | None = None) -> np.ndarray:
    """Apply ``ops`` (objects with ``.targets`` and ``.matrix``) in order."""
    if psi is None:
        psi = zero_state(n)
    for op in ops:
        apply(psi, op.targets, op.matrix)
    return psi


def probabilities(psi: np.ndarray) -> np.ndarray:
    n = int(psi.size).bit_length() - 1
    p = np.empty(psi.size, dtype=np.float64)
    lib().orc_probabilities(_dptr(np.ascontiguousarray(psi).view(np.float64)), n, _dptr(p))
    return p


def expect_z(psi: np.ndarray, mask: int) -> float:
    n = int(psi.size).bit_length() - 1
    return float(lib().orc_expect_z(_dptr(np.ascontiguousarray(psi).view(np.float64)), n, ctypes.c_uint64(mask)))


def philox4x64_10(ctr: Sequence[int], key: Sequence[int]) -> List[int]:
    c = (ctypes.c_uint64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (ctypes.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(v) for v in o]


def sample(psi_logical: np.ndarray, phys_of_logical: Sequence[int], shots: int, seed: int, stream: int = 0,
           near_frac: float = 0.0) -> Tuple[np.ndarray, np.ndarray]:
    """Per-shot logical outcomes and near-boundary flags (see qsa_oracle.c)."""
    psi = np.ascontiguousarray(psi_logical, dtype=np.complex128)
    n = int(psi.size).bit_length() - 1
    lay = (ctypes.c_int * n)(*[int(v) for v in phys_of_logical])
    out = np.empty(shots, dtype=np.uint64)
    flg = np.empty(shots, dtype=np.uint8)
    rc = lib().orc_sample(_dptr(psi.view(np.float64)), n, lay, shots, seed, stream, near_frac,
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                          flg.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if rc != 0:
        raise ValueError("oracle sample: all weights are zero")
    return out, flg.astype(bool)


def sample_counts(psi_logical, phys_of_logical, shots, seed, stream=0):
    out, _ = sample(psi_logical, phys_of_logical, shots, seed, stream)
    vals, cnts = np.unique(out, return_counts=True)
    return vals.astype(np.uint64), cnts.astype(np.uint64)


# ---------------------------------------------------------------------------
# Independent full-matrix construction (for pins at N <= 8)
# ---------------------------------------------------------------------------

def full_operator(n: int, targets: Sequence[int], mat: np.ndarray) -> np.ndarray:
    """The 2^n x 2^n operator of ``mat`` on ``targets`` built as
    P^T (I_{2^(n-k)} kron G) P, where P is the basis permutation that moves
    qubit q_j to bit j and the remaining qubits, in increasing order, to bits
    k..n-1.  Built from np.kron and an explicit permutation matrix, not from
    the gather/scatter loop of ``apply``."""
    k = len(targets)
    rest = [q for q in range(n) if q not in targets]
    order = list(targets) + rest  # new bit i holds old qubit order[i]
    dim = 1 << n
    P = np.zeros((dim, dim))
    for x in range(dim):
        y = 0
        for i, q in enumerate(order):
            if (x >> q) & 1:
                y |= 1 << i
        P[y, x] = 1.0
    big = np.kron(np.eye(1 << (n - k)), np.asarray(mat, dtype=np.complex128))
    return P.T @ big @ P


# ---------------------------------------------------------------------------
# Fusion: embedding, block product, partitions (§IV-C)
# ---------------------------------------------------------------------------

def kron_embed(mat: np.ndarray, gate_targets: Sequence[int], block_targets: Sequence[int]) -> np.ndarray:
    """Matrix of a gate on ``gate_targets`` as an operator on the ordered
    tuple ``block_targets`` (⊇ gate_targets), entry by entry from the
    definition: E[r][c] = G[r_g][c_g] when r and c agree on every block bit
    that is not a gate target, else 0, where r_g collects the bits of r at the
    block positions of the gate's targets, in the gate's order."""
    u = len(block_targets)
    pos = [list(block_targets).index(q) for q in gate_targets]
    other = [i for i in range(u) if i not in pos]
    D = 1 << u
    E = np.zeros((D, D), dtype=np.complex128)
    for r in range(D):
        for c in range(D):
            if any(((r >> i) & 1) != ((c >> i) & 1) for i in other):
                continue
            rg = sum(((r >> p) & 1) << j for j, p in enumerate(pos))
            cg = sum(((c >> p) & 1) << j for j, p in enumerate(pos))
            E[r, c] = mat[rg, cg]
    return E


def block_product(gates: Sequence, block_targets: Sequence[int]) -> np.ndarray:
    """Product of the gates of one block in circuit order, later gates on the
    left (§IV-C)."""
    D = 1 << len(block_targets)
    M = np.eye(D, dtype=np.complex128)
    for g in gates:
        M = kron_embed(g.matrix, g.targets, block_targets) @ M
    return M


def gamma_score(width: int, diag: bool, prod: bool = False) -> float:
    """gamma(k, dense) = 4^k, gamma(k, diag) = 1 (§IV-C); a product block (one
    streaming pass, like a diagonal one) also scores 1."""
    return 1.0 if (diag or prod) else float(4 ** width)


def _block_width(gates, j, i):
    s = set()
    for g in gates[j:i]:
        s.update(g.targets)
    return len(s)


def dp_window(gates: Sequence, kmax: int, kmax_diag: int, score=None) -> List[Tuple[int, int]]:
    """Eq. dp-recurrence on one window g_0..g_{h-1}:
        D_0 = 0,  D_i = min_{j in J_i} D_j + Gamma(B(j, i)),
    J_i = {j < i : width(B(j,i)) <= cap(mode(B(j,i)))} ∪ {i-1}.  Ties take the
    smallest j (longest final block).  Returns the blocks as (start, end)
    half-open gate ranges, in order.  ``score(width, diag, gates_slice)``
    replaces Gamma when given."""
    h = len(gates)
    INF = float("inf")
    D = [0.0] + [INF] * h
    arg = [0] * (h + 1)
    for i in range(1, h + 1):
        best, bj = INF, None
        for j in range(0, i):
            blk = gates[j:i]
            w = _block_width(gates, j, i)
            diag = all(g.diag for g in blk)
            prod = i - j == 1 and getattr(blk[0], "prod", False)
            cap = kmax_diag if diag else kmax
            if w > cap and j != i - 1:
                continue
            sc = gamma_score(w, diag, prod) if score is None else score(w, diag, blk)
            val = D[j] + sc
            if val < best:  # strict: keeps the smallest j on ties
                best, bj = val, j
        D[i], arg[i] = best, bj
    blocks = []
    i = h
    while i > 0:
        j = arg[i]
        blocks.append((j, i))
        i = j
    return blocks[::-1]


def greedy_partition(gates: Sequence, kmax: int) -> List[Tuple[int, int]]:
    """Plain width-limit heuristic: walk the gates in circuit order and extend
    the current block while the union of targets stays within kmax; otherwise
    close it.  A gate wider than kmax is a singleton."""
    blocks = []
    start, cur = 0, set()
    for i, g in enumerate(gates):
        nxt = cur | set(g.targets)
        if i > start and len(nxt) > kmax:
            blocks.append((start, i))
            start, cur = i, set(g.targets)
        else:
            cur = nxt
    if gates:
        blocks.append((start, len(gates)))
    return blocks


# ---------------------------------------------------------------------------
# Cost-model network (FP64): 37 -> 64 -> ReLU -> 64 -> ReLU -> 1
# ---------------------------------------------------------------------------

MLP_SHAPES = [(64, 37), (64,), (64, 64), (64,), (1, 64), (1,)]


def mlp_forward(params: Sequence[np.ndarray], X: np.ndarray):
    """y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for each row x of X."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3.T + b3
    return y[:, 0], (X, z1, a1, z2, a2)


def mlp_loss_grad(params, X, t):
    """L = mean((y - t)^2); returns L and dL/dparams by the chain rule."""
    W1, b1, W2, b2, W3, b3 = params
    y, (X, z1, a1, z2, a2) = mlp_forward(params, X)
    n = X.shape[0]
    L = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / n                  # (n,)
    dW3 = dy[None, :] @ a2                   # (1,64)
    db3 = np.array([dy.sum()])
    da2 = dy[:, None] * W3                   # (n,64)
    dz2 = da2 * (z2 > 0)
    dW2 = dz2.T @ a1
    db2 = dz2.sum(axis=0)
    da1 = dz2 @ W2
    dz1 = da1 * (z1 > 0)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    return L, [dW1, db1, dW2, db2, dW3, db3]


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), step number t >= 1."""
    new_p, new_m, new_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = b1 * mm + (1 - b1) * g
        vv = b2 * vv + (1 - b2) * g * g
        mh = mm / (1 - b1 ** t)
        vh = vv / (1 - b2 ** t)
        new_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        new_m.append(mm)
        new_v.append(vv)
    return new_p, new_m, new_v


# ---------------------------------------------------------------------------
# Fidelity metrics
# ---------------------------------------------------------------------------

def fidelity(psi_ref: np.ndarray, psi: np.ndarray) -> float:
    """F = |<psi_ref|psi>|^2 in FP64."""
    a = np.asarray(psi_ref, dtype=np.complex128)
    b = np.asarray(psi, dtype=np.complex128)
    return float(abs(np.vdot(a, b)) ** 2)


def max_abs_diff(psi_ref: np.ndarray, psi: np.ndarray) -> float:
    return float(np.max(np.abs(np.asarray(psi_ref, np.complex128) - np.asarray(psi, np.complex128))))


# ---------------------------------------------------------------------------
# Layout map (§II, §IV-B Alg. 2, §IV-D Theorem 1)
# ---------------------------------------------------------------------------

def decode_state(stored: np.ndarray, phys_of_logical: Sequence[int]) -> np.ndarray:
    """Canonical logical state from a stored one: psi_x = stored[y] with
    y_{L(q)} = x_q for every logical qubit q (Theorem 1, component form)."""
    n = int(stored.size).bit_length() - 1
    x = np.arange(stored.size, dtype=np.uint64)
    y = np.zeros_like(x)
    for q in range(n):
        y |= ((x >> np.uint64(q)) & np.uint64(1)) << np.uint64(phys_of_logical[q])
    return stored[y]


def encode_state(psi: np.ndarray, phys_of_logical: Sequence[int]) -> np.ndarray:
    """Inverse of decode_state: stored[y] = psi_x with y_{L(q)} = x_q."""
    n = int(psi.size).bit_length() - 1
    x = np.arange(psi.size, dtype=np.uint64)
    y = np.zeros_like(x)
    for q in range(n):
        y |= ((x >> np.uint64(q)) & np.uint64(1)) << np.uint64(phys_of_logical[q])
    out = np.empty_like(psi)
    out[y] = psi
    return out


def lazy_ttgt(stored: np.ndarray, phys_of_logical: Sequence[int], targets: Sequence[int], mat: np.ndarray):
    """Dense branch of Alg. 2 (lazy TTGT), out of place:
    A = (L(q_0)..L(q_{k-1})); alpha_A sends A_j to position N-k+j and the
    other positions, in increasing order, to 0..N-k-1; the data permutation
    Pi_A moves bit b of every index to bit alpha_A(b); the result is viewed
    as M (2^k x 2^(N-k), row = the top k bits), M' = G M, and L' = alpha_A∘L.
    Returns (L', stored')."""
    n = int(stored.size).bit_length() - 1
    k = len(targets)
    A = [phys_of_logical[q] for q in targets]
    alpha = {}
    for j, b in enumerate(A):
        alpha[b] = n - k + j
    rest = [b for b in range(n) if b not in A]
    for i, b in enumerate(rest):
        alpha[b] = i
    y = np.arange(stored.size, dtype=np.uint64)
    yp = np.zeros_like(y)
    for b in range(n):
        yp |= ((y >> np.uint64(b)) & np.uint64(1)) << np.uint64(alpha[b])
    perm = np.empty_like(stored)
    perm[yp] = stored
    M = perm.reshape(1 << k, 1 << (n - k))
    Mp = np.asarray(mat, dtype=np.complex128) @ M
    Lp = [alpha[phys_of_logical[q]] for q in range(n)]
    return Lp, Mp.reshape(-1).copy()


def promotion_replay(tuples: Sequence[Sequence[int]], n: int, frames: int, policy: str,
                     layout: Sequence[int] | None = None, history: bool = False):
    """Replay of on-demand promotions over a fused stream (§IV-D, Corollary
    "ideal minimal demand-promotion count"): the ``frames`` lowest physical
    positions are page frames, logical qubits are pages.  Before tuple i, each
    of its targets (in tuple order) that is not in a frame is promoted by
    swapping its position with a victim frame that holds no target of tuple i
    (and was not filled for it already).  ``policy``: ``"first_free"`` takes
    the lowest such frame (the CPU-MPI rule); ``"farthest"`` takes the frame
    whose qubit is next targeted farthest in the future (never = infinity),
    ties to the lowest frame (Belady).  Returns (promotions per tuple, final
    layout phys_of_logical), plus the layout each tuple ran under when
    ``history``."""
    L = list(range(n)) if layout is None else [int(v) for v in layout]
    inv = [0] * n
    for q, p in enumerate(L):
        inv[p] = q
    counts, hist = [], []
    for i, tup in enumerate(tuples):
        pinned = {L[q] for q in tup if L[q] < frames}
        c = 0
        for q in tup:
            if L[q] < frames:
                continue
            cand = [p for p in range(frames) if p not in pinned]
            if not cand:
                raise ValueError("tuple wider than the frames")
            if policy == "first_free":
                v = cand[0]
            elif policy == "farthest":
                def next_use(p):
                    qq = inv[p]
                    for j in range(i + 1, len(tuples)):
                        if qq in tuples[j]:
                            return j
                    return float("inf")
                best = max(next_use(p) for p in cand)
                v = min(p for p in cand if next_use(p) == best)
            else:
                raise ValueError(policy)
            hp, qv = L[q], inv[v]
            L[q], L[qv] = v, hp
            inv[v], inv[hp] = q, qv
            pinned.add(v)
            c += 1
        counts.append(c)
        if history:
            hist.append(list(L))
    return (counts, L, hist) if history else (counts, L)


def merge_adjacent(blocks, kmax: int, kmax_diag: int, score=None):
    """Cross-window greedy merge (§IV-C, reading: merge neighbours a, b when
    width(a ∪ b) fits the cap of the merged mode and
    Gamma(a ∪ b) <= Gamma(a) + Gamma(b)).  ``blocks`` are dicts with keys
    targets (set), diag, s, e (input op range)."""
    def sc(blk):
        if score is None:
            return gamma_score(len(blk["targets"]), blk["diag"], blk.get("prod", False))
        return score(len(blk["targets"]), blk["diag"], blk["targets"])

    out = []
    cur = None
    for b in blocks:
        if cur is None:
            cur = dict(b)
            continue
        t = cur["targets"] | b["targets"]
        d = cur["diag"] and b["diag"]
        cap = kmax_diag if d else kmax
        merged = {"targets": t, "diag": d, "s": cur["s"], "e": b["e"], "prod": False}
        if len(t) <= cap and sc(merged) <= sc(cur) + sc(b):
            cur = merged
        else:
            out.append(cur)
            cur = dict(b)
    if cur is not None:
        out.append(cur)
    return out


def fuse_pipeline(gates, kmax: int, kmax_diag: int, window: int = 64, rounds: int = 4, score=None):
    """Windows of ``window`` units partitioned by Eq. dp-recurrence, then the
    cross-window merge; the pipeline is repeated on the resulting blocks at
    most ``rounds`` times and stops when the block count no longer falls
    (§IV-C).  Returns the first input-op index of every block."""

    class U:
        def __init__(self, targets, diag, s, e, prod=False):
            self.targets, self.diag, self.s, self.e = tuple(sorted(targets)), diag, s, e
            self.prod = prod

    units = [U(g.targets, bool(g.diag), i, i + 1, bool(getattr(g, "prod", False))) for i, g in enumerate(gates)]
    wscore = None if score is None else (lambda w, d, blk: score(w, d, set().union(*[set(b.targets) for b in blk])))
    for rnd in range(rounds):
        blocks = []
        for b0 in range(0, len(units), window):
            win = units[b0:b0 + window]
            for j, i in dp_window(win, kmax, kmax_diag, score=wscore):
                t = set()
                for u in win[j:i]:
                    t |= set(u.targets)
                blocks.append({"targets": t, "diag": all(u.diag for u in win[j:i]), "s": win[j].s,
                               "e": win[i - 1].e, "prod": i - j == 1 and win[j].prod})
        blocks = merge_adjacent(blocks, kmax, kmax_diag, score)
        if rnd > 0 and len(blocks) >= len(units):
            break
        units = [U(b["targets"], b["diag"], b["s"], b["e"], b.get("prod", False)) for b in blocks]
    return [u.s for u in units]


def fuse_pipeline_products(ops, kmax: int, kmax_diag: int, kmax_prod: int, window: int = 64, rounds: int = 4):
    """The fusion pipeline over product units (:func:`product_units`): a unit
    of two or more qubits is a product unit, scored as one pass while it
    stays a block of its own; merged with other units it becomes dense.
    Returns the first op index of every block."""

    class G:
        def __init__(self, targets, prod):
            self.targets, self.diag, self.prod = tuple(sorted(targets)), False, prod

    units = product_units(ops, kmax_prod)
    gates = []
    for a, b in units:
        t = sorted({int(q) for o in ops[a:b] for q in o.targets})
        if b - a == 1:
            gates.append(ops[a])
        else:
            gates.append(G(t, len(t) >= 2))
    starts = fuse_pipeline(gates, kmax, kmax_diag, window, rounds)
    return [units[i][0] for i in starts]

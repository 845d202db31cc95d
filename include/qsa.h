/*
 * qsa.h — C ABI of libqsa, a GB300 (sm_103a) state-vector library that applies
 * ordered fused k-qubit operators (k = 1..6) to a complex64 state vector whose
 * qubits are placed by a logical-to-physical layout map.
 *
 * Paper: "QSimAdv" (arxiv 2608.16940).  Cited passages:
 *   §II   "State and layout notation", "Fused gates and requests"
 *   §III  (R2) apply(L, Psi, G, V) -> (L', Psi')
 *   §IV-B Alg. 2 (axis-shifted / lazy-TTGT lowering), Eqs. cost-perm, cost-formal
 *   §IV-C fusion score gamma, Eq. dp-recurrence, window W = 64, cross-window merge
 *   §IV-D Theorem 1 (placement invariant), Alg. 3 (promotion dispatch), first-free
 *   §IV-E "Sampling" (hierarchical CDF, strict upper bound), App. B numerics
 *
 * Conventions shared by every call
 *   - A state of N qubits holds 2^N amplitudes; amplitude y is stored as two
 *     floats (Re, Im) at byte offset 8*y of one device buffer.  Bit p of y is
 *     physical position p, position 0 least significant (§II).
 *   - The layout map L sends logical qubit q to physical position L(q); it is
 *     a bijection on 0..N-1.  The stored amplitude at y equals the logical one
 *     at x with x_q = y_{L(q)} (Theorem 1).  New states have L = identity.
 *   - A k-qubit matrix G acts on the ordered logical tuple V = (q_0..q_{k-1});
 *     q_j supplies bit j of G's row and column index (little-endian in V, §II).
 *     Matrices are passed as 2*4^k doubles, row-major G[r][c], interleaved
 *     (Re, Im); the library rounds them once to FP32.
 *   - Host pointers are read before the call returns (the caller keeps
 *     ownership).  Device pointers are borrowed, never freed by the library.
 *   - Kernels run on the state's CUDA stream (a cudaStream_t passed as void*;
 *     NULL = legacy default stream).  apply / permute calls are asynchronous;
 *     calls that return numbers to host memory synchronise that stream.
 *   - Every call returns qsa_status; on failure qsa_last_error() gives a
 *     message (thread-local).  Arguments are validated before any launch.
 *     After QSA_E_CUDA the state is marked failed and later calls on it
 *     return QSA_E_STATE.
 */
#ifndef QSA_H
#define QSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QSA_OK = 0,
    QSA_E_ARG = 1,          /* invalid argument (range, duplicate target, NULL, non-bijection) */
    QSA_E_RANGE = 2,        /* output capacity too small; the needed size is reported */
    QSA_E_NOMEM = 3,        /* device allocation failed */
    QSA_E_CUDA = 4,         /* a CUDA call or kernel failed; the state is marked failed */
    QSA_E_TIMEOUT = 5,      /* a device-side work budget ran out (the kernel returned early) */
    QSA_E_UNSUPPORTED = 6,  /* valid request this build does not implement (e.g. complex128) */
    QSA_E_STATE = 7         /* call not allowed in the state's current condition */
} qsa_status;

typedef enum { QSA_C64 = 0, QSA_C128 = 1 /* reserved: QSA_E_UNSUPPORTED */ } qsa_dtype;

typedef struct qsa_state_s* qsa_state;

#define QSA_MAX_QUBITS 34
#define QSA_MAX_K 6
/* Widest diagonal operator (qsa_apply_diag, diagonal plan blocks).  The
 * paper caps marked-diagonal blocks at 6 on GPU (App. "Fusion
 * configuration"); the streaming kernel keeps its 2^k-entry table in shared
 * memory, so this build accepts up to 12. */
#define QSA_MAX_DIAG 12
/* Widest product block (qsa_apply_product, product plan blocks): one-qubit
 * factors on distinct qubits, applied in one pass of the FP32 tile engine
 * (2^11-amplitude tiles) when at most 6 of them lie above the tile's
 * contiguous low bits, else in several passes. */
#define QSA_MAX_PROD 11
/* Layer blocks (qsa_apply_layer, layer plan blocks): tiles of 2^12
 * amplitudes whose 3 lowest bits are the state's 3 lowest positions, so at
 * most 9 factor positions may lie at 3 or above; up to 12 factors. */
#define QSA_LAYER_TILE_BITS 12
#define QSA_LAYER_LOW_BITS 3
#define QSA_MAX_LAYER 12

/* Lowering of one fused dense operator (§III R4: the backend picks the
 * concrete kernel once the physical targets are known). */
typedef enum {
    QSA_LOWER_AUTO = 0,     /* strided in-place gather unless the cost model says otherwise */
    QSA_LOWER_STRIDED = 1,  /* gather the 2^k group straight from any physical positions */
    QSA_LOWER_PERMUTE = 2   /* first promote targets outside the in-block bits by bit swaps
                               (first-free victims, §IV-D), keep the new layout, then apply */
} qsa_lowering;

typedef enum {
    QSA_PREC_FP32 = 0,      /* FP32 CUDA-core complex matvec */
    QSA_PREC_TF32X3 = 1     /* k = 5, 6: split-TF32 (3 products) on tcgen05 tensor cores with
                               FP32 accumulation; k < 5 falls back to FP32 */
} qsa_precision;

typedef enum {
    QSA_PLAN_PER_GATE = 0,  /* no fusion: one pass per input op */
    QSA_PLAN_GREEDY = 1,    /* width-limit greedy in circuit order */
    QSA_PLAN_DP = 2,        /* Eq. dp-recurrence with gamma = 4^k (dense) / 1 (diag) */
    QSA_PLAN_DP_MLP = 3     /* the same DP scored by the cost model's predicted seconds;
                               falls back to QSA_PLAN_GREEDY when no model is loaded */
} qsa_planner;

#define QSA_OP_DIAG 1u      /* op is diagonal (eligible for the diagonal block mode, §IV-C) */

/* One circuit operation: G on the ordered logical targets[0..k-1]. */
typedef struct {
    int32_t k;              /* 1..6 */
    int32_t targets[QSA_MAX_K];
    const double* matrix;   /* host, 2*4^k doubles, layout as above */
    uint32_t flags;         /* QSA_OP_DIAG or 0 */
} qsa_op;

/* Which in-block position a promotion evicts (§IV-D).  The frames are the
 * min(11, N) lowest physical positions (the in-block bits of the tile). */
typedef enum {
    QSA_VICTIM_FIRST_FREE = 0,  /* lowest position not holding a target of the block (the CPU-MPI rule) */
    QSA_VICTIM_FARTHEST = 1     /* position whose qubit a later dense block of the plan targets farthest
                                   in the future (never = infinity), ties to the lowest; Corollary
                                   "ideal minimal demand-promotion count" (Belady) */
} qsa_victim;

typedef struct {
    int32_t planner;        /* qsa_planner */
    int32_t kmax;           /* dense fusion cap, 1..6 */
    int32_t kmax_diag;      /* diagonal-block cap, 1..QSA_MAX_DIAG (independent of kmax;
                               the batch path needs kmax_diag <= kmax) */
    int32_t window;         /* DP window W (§IV-C uses 64) */
    int32_t rounds;         /* fuse pipeline repeats, 1..4 (§IV-C: at most four) */
    int32_t precision;      /* qsa_precision for k >= 5 blocks */
    int32_t lowering;       /* qsa_lowering */
    int32_t timing;         /* 1: time every launch with CUDA events (fills *_seconds) */
    int32_t victim;         /* qsa_victim: eviction rule of QSA_LOWER_PERMUTE promotions */
    int32_t kmax_prod;      /* 0 or 1: off; 2..QSA_MAX_PROD: maximal runs of non-diagonal one-qubit ops
                               on at most this many qubits become product units, applied as one product
                               block (one pass) while they stay blocks of their own (§IV-D structured
                               blocks); not used by per-gate plans or batches */
    int32_t layer;          /* 1: group the circuit into layer units first (qsa_apply_layer: one- and
                               two-qubit QSA_OP_DIAG ops, then one-qubit ops on qubits whose positions
                               fit a tile), moving ops only across ops they commute with (lookahead 256
                               skipped ops); a layer unit runs as one layer block while it stays a block
                               of its own.  Replaces kmax_prod.  0: off.  Not used by batches */
    int32_t zero_init;      /* 1: the plan runs on |0..0> (the state must be known zero when it starts,
                               else QSA_E_STATE).  Its prefix of one-qubit ops, each on a qubit no
                               earlier diagonal gate of the prefix touches, and diagonal gates on at most
                               two qubits leaves prod_q a_q[x_q] * prod_g d_g(x) (a_q: the qubit's ops
                               applied to |0>), written in one write-only pass (§IV-D: |0..0> is the
                               state whose relabelling is free; here its evolution by a product of
                               one-qubit ops is too).  0: off.  Not used by batches */
} qsa_plan_opts;

typedef struct {
    double seconds;         /* device time of all launches (timing = 1), else 0 */
    double apply_seconds;   /* device time of FP32 fused-operator kernels */
    double permute_seconds; /* device time of permutation kernels */
    double hbm_bytes;       /* algorithmic HBM bytes: 16 B x 2^N per full-state pass */
    uint64_t blocks;        /* fused blocks applied */
    uint64_t passes;        /* full-state passes (applies + permutations) */
    uint64_t permutes;      /* permutation passes */
    uint64_t tc_blocks;     /* blocks run on the tensor-core path */
    uint64_t launches;      /* kernel launches issued */
    double h2d_bytes;       /* host-to-device bytes copied by the call (fused matrices) */
    double tc_seconds;      /* device time of tensor-core fused-operator kernels */
    uint64_t diag_blocks;   /* diagonal blocks run on the streaming kernel */
    double diag_seconds;    /* device time of diagonal streaming kernels */
    uint64_t prod_blocks;   /* product blocks (one-qubit factors) applied */
    double prod_seconds;    /* device time of product kernels */
    uint64_t layer_blocks;  /* layer blocks applied */
    double layer_seconds;   /* device time of layer passes (their per-tile record kernels excluded) */
} qsa_run_stats;

/* A compiled circuit: the planner's blocks with their fused FP32 matrices. */
typedef struct qsa_plan_s* qsa_plan;

/* ---- state lifecycle (§II; §III R2) ---------------------------------------- */

/* Allocate a 2^N-amplitude state (library-owned device memory) set to |0..0>
 * with identity layout, on the legacy default stream.  N in 1..34.
 * Errors: QSA_E_ARG (N, out NULL), QSA_E_UNSUPPORTED (dtype != QSA_C64),
 * QSA_E_NOMEM. */
qsa_status qsa_state_create(int n_qubits, qsa_dtype dtype, qsa_state* out);

/* Wrap a caller-owned device buffer of >= 8*2^N bytes (16-byte aligned) that
 * must outlive the state.  init_zero = 1 writes |0..0>; 0 keeps the buffer's
 * contents as the initial stored state (identity layout).  cuda_stream is
 * the stream all kernels of this state run on. */
qsa_status qsa_state_create_ex(int n_qubits, qsa_dtype dtype, void* dev_buf, size_t bytes,
                               void* cuda_stream, int init_zero, qsa_state* out);

/* Free library-owned memory and the handle (synchronises its stream). */
qsa_status qsa_state_destroy(qsa_state s);

/* Change the stream used by later calls. */
qsa_status qsa_set_stream(qsa_state s, void* cuda_stream);

/* |0..0> and identity layout (clears a failed mark only if the device is healthy). */
qsa_status qsa_state_reset(qsa_state s);

/* Number of qubits, and the device address of the amplitudes. */
qsa_status qsa_state_info(qsa_state s, int* n_qubits, void** dev_amplitudes);

/* ---- layout map (§II, §IV-D Theorem 1) ------------------------------------- */

/* Install layout phys_of_logical[q] = L(q) (N entries, a bijection, else
 * QSA_E_ARG).  materialise = 1 moves the amplitudes so the logical state is
 * unchanged (permutation passes).  materialise = 0 only relabels, which is
 * valid only while the state is known to be |0..0> (§IV-D: a metadata-only
 * relabel is valid for the permutation-invariant initial state); otherwise
 * QSA_E_STATE. */
qsa_status qsa_set_layout(qsa_state s, const int32_t* phys_of_logical, int materialise);

/* Copy the current layout into phys_of_logical[0..N-1]. */
qsa_status qsa_get_layout(qsa_state s, int32_t* phys_of_logical);

/* The qubit-permutation kernel (single-GPU promotion, Alg. 3 with rank bits
 * read as out-of-block bits; Lemma "distributed promotion swap"): swap
 * physical bit positions phys_a[i] <-> phys_b[i] for i < n_pairs in place and
 * compose the layout with the same transpositions.  Positions must be
 * distinct across all pairs (QSA_E_ARG).  Pure data movement: bit-exact. */
qsa_status qsa_permute_bits(qsa_state s, const int32_t* phys_a, const int32_t* phys_b, int n_pairs);

/* ---- fused operator (§III R2, Alg. 2) --------------------------------------- */

/* apply(L, Psi, G, V) -> (L', Psi'): resolve A = (L(q_0)..L(q_{k-1})) and
 * apply G in V's little-endian order.  targets: k distinct logical qubits
 * (host); matrix: host, 2*4^k doubles.  Uses QSA_LOWER_AUTO and FP32.
 * Errors: QSA_E_ARG (k outside 1..6 or > N, bad / repeated target, NULL). */
qsa_status qsa_apply_fused(qsa_state s, const int32_t* targets, int k, const double* matrix);

/* As qsa_apply_fused with an explicit lowering (qsa_lowering) and precision
 * (qsa_precision).  QSA_LOWER_PERMUTE may change the layout (L' = tau o L). */
qsa_status qsa_apply_fused_ex(qsa_state s, const int32_t* targets, int k, const double* matrix,
                              int lowering, int precision);

/* Diagonal branch of Alg. 2 (Eq. cost-diag-formal: one streaming pass, no
 * permutation): psi[y] <- diag[c] * psi[y], where bit j of c is bit L(q_j)
 * of the physical index y; the layout is unchanged.  targets: k distinct
 * logical qubits (host); diag: host, 2 * 2^k doubles, entry c as (Re, Im),
 * rounded once to FP32.  Any complex entries are accepted (not only phases).
 * Errors: QSA_E_ARG (k outside 1..QSA_MAX_DIAG or > N, bad / repeated
 * target, NULL). */
qsa_status qsa_apply_diag(qsa_state s, const int32_t* targets, int k, const double* diag);

/* Product operator U_{k-1} (x) ... (x) U_0 with the 2x2 factor U_j on logical
 * qubit targets[j]: a structured fused block (§IV-D: structured blocks may use
 * cheaper lowerings), applied in one pass of the tile engine with 2k complex
 * multiply-adds per amplitude instead of 2^k (several passes when more than 6
 * targets lie above the tile's contiguous low bits).  targets: k distinct
 * logical qubits (host); factors: host, 8 doubles per factor (row-major 2x2,
 * interleaved Re, Im), rounded once to FP32.  The layout is unchanged.
 * Errors: QSA_E_ARG (k outside 1..QSA_MAX_PROD or > N, bad / repeated target,
 * NULL). */
qsa_status qsa_apply_product(qsa_state s, const int32_t* targets, int k, const double* factors);

/* Layer block: every diagonal op diag_ops[0..n_diag) (k = 1 or 2, diagonal
 * matrix; off-diagonal entries must be zero), then the product of the 2x2
 * factor j on logical qubit targets[j] (distinct qubits; a diagonal op may
 * share qubits with factors, it acts first) -- a structured fused block
 * (§IV-D), in one pass when N >= 12 and at most QSA_LAYER_TILE_BITS -
 * QSA_LAYER_LOW_BITS factor positions lie at QSA_LAYER_LOW_BITS or above
 * (else the factors are split over several passes, the diagonal ops in the
 * first).  Per tile of 2^12 amplitudes the diagonal ops become a 2^12-entry
 * table over the tile's bits (ops with every qubit in the tile), one-qubit
 * phases folded into the factors (ops with one qubit in the tile) and a scalar
 * (ops with none), so any number of them costs one pass.  Matrices and
 * factors are rounded once to FP32 (tables formed in FP64).  factors: host,
 * 8 doubles per factor (row-major 2x2, interleaved Re, Im); k = 0 applies the
 * diagonal ops only.  N < 12 runs the ops on the diagonal and product kernels.
 * The layout is unchanged.  Errors: QSA_E_ARG (k outside 0..QSA_MAX_LAYER or
 * > N, bad / repeated target, a diagonal op that is not k = 1, 2 or not
 * diagonal, NULL). */
qsa_status qsa_apply_layer(qsa_state s, const qsa_op* diag_ops, size_t n_diag, const int32_t* targets, int k,
                           const double* factors);

/* ---- density matrices (§IV-B density-matrix wrapper) ----------------------- */

/* An n-qubit density matrix (2 <= n <= 17) is held as a 2n-qubit state
 * (qsa_state_create(2n, ...)): vec(rho) stacked column-major, index
 * row + 2^n * column, so the lower n qubits are row bits and qubit q + n is
 * the column copy of qubit q; the state's |0..0> is |0..0><0..0|.  The state
 * keeps its own layout map; the calls below resolve through it. */

/* Host only: lower a k-qubit channel {E_i} of an n-qubit density matrix to
 * one 2k-qubit operator of the vectorised state, so that channels and gates
 * enter qsa_plan_create / qsa_apply_circuit as ordinary fused operators:
 * targets_out (2k entries) = (targets, targets + n) -- row copies first, then
 * column copies, target order kept in each group; matrix_out (2 * 16^k
 * doubles, the qsa_op layout) = sum_i conj(E_i) (x) E_i with E_i on the row
 * bits (index bits 0..k-1) and conj(E_i) on the column bits, summed in FP64.
 * kraus: n_kraus x 2 * 4^k doubles (each E_i row-major, interleaved Re, Im).
 * Errors: QSA_E_ARG (n outside 2..17, k outside 1..3, targets, n_kraus < 1,
 * NULL). */
qsa_status qsa_dm_superoperator(int n, const int32_t* targets, int k, const double* kraus, int n_kraus,
                                int32_t* targets_out, double* matrix_out);

/* rho <- sum_i E_i rho E_i^dagger: the superoperator sum_i conj(E_i) (x) E_i
 * (formed once in FP64 on the host) applied as one fused 2k-qubit operator at
 * (targets, targets + n) -- row copies first, original factor on the row
 * bits -- through the dense path (precision: qsa_precision for 2k = 6).  A
 * unitary is the one-operator channel.  targets: k distinct qubits of the
 * density matrix (host), k in 1..3; kraus: host, n_kraus x 2 * 4^k doubles
 * (each E_i row-major, interleaved Re, Im).  Trace preservation is the
 * caller's (it is not checked).  Errors: QSA_E_ARG (state not 2n qubits,
 * n outside 2..17, k, targets, n_kraus < 1, NULL). */
qsa_status qsa_dm_apply_channel(qsa_state s, int n, const int32_t* targets, int k, const double* kraus,
                                int n_kraus, int precision);

/* Diagonal of rho: out_host (host, 2^n doubles, nullable) receives rho_xx in
 * logical order (real parts, FP32 data summed in FP64); *trace_out (nullable)
 * the sum.  Synchronises the stream.  Errors: QSA_E_ARG, QSA_E_NOMEM. */
qsa_status qsa_dm_probabilities(qsa_state s, int n, double* out_host, double* trace_out);

/* Tr(rho Z_mask) = sum_x rho_xx (-1)^popc(x & mask) over the density matrix's
 * qubits (mask < 2^n), reduced in FP64 on the GPU.  Synchronises the stream. */
qsa_status qsa_dm_expectation_z(qsa_state s, int n, uint64_t mask, double* out);

/* ---- circuits: fusion planning + execution (§IV-C) ------------------------- */

/* Fill *opts with the defaults: DP planner, kmax 4, kmax_diag 4, window 64,
 * rounds 4, FP32, AUTO lowering, timing off. */
void qsa_plan_opts_default(qsa_plan_opts* opts);

/* Host only (no GPU needed): partition ops[0..n_ops-1] into consecutive
 * fused blocks with the planner in *opts (NULL = defaults).  block_start
 * receives the first op index of each block (capacity n_ops entries);
 * *n_blocks the number of blocks.  Blocks may cover several input ops after
 * the merge / repeat rounds.  Errors: QSA_E_ARG. */
qsa_status qsa_plan_circuit(const qsa_op* ops, size_t n_ops, int n_qubits, const qsa_plan_opts* opts,
                            size_t* block_start, size_t* n_blocks);

/* Host only: the fused matrix of ops[0..n_ops-1] in circuit order (later ops
 * multiplied on the left, §IV-C), on the ordered logical tuple
 * block_targets_out (the union of the ops' targets, ascending; at most 6).
 * matrix_out: 2*4^u doubles.  *width_out = u.  Errors: QSA_E_ARG (union > 6). */
qsa_status qsa_fuse_ops(const qsa_op* ops, size_t n_ops, int32_t* block_targets_out, int* width_out,
                        double* matrix_out);

/* Plan (as qsa_plan_circuit), fuse and apply the circuit to s.  stats may be
 * NULL.  With opts->timing = 1 the call synchronises at the end and fills the
 * device times.  Equivalent to qsa_plan_create + qsa_plan_execute +
 * qsa_plan_destroy with the state's current layout. */
qsa_status qsa_apply_circuit(qsa_state s, const qsa_op* ops, size_t n_ops, const qsa_plan_opts* opts,
                             qsa_run_stats* stats);

/* Host only: plan and fuse once (§IV-C; the paper's timer excludes plan
 * construction, App. B).  layout (N entries, nullable = identity) is the
 * layout the DP-MLP scores assume.  The plan copies everything it needs from
 * ops.  Errors: as qsa_plan_circuit. */
qsa_status qsa_plan_create(const qsa_op* ops, size_t n_ops, int n_qubits, const qsa_plan_opts* opts,
                           const int32_t* layout, qsa_plan* out);

/* Number of fused blocks and input ops, widest block, bytes of fused FP32 matrices. */
qsa_status qsa_plan_info(qsa_plan p, size_t* n_blocks, size_t* n_ops, int* max_width, size_t* matrix_bytes);

/* First input op and width of every block (capacity >= n_blocks, else QSA_E_RANGE). */
qsa_status qsa_plan_blocks(qsa_plan p, size_t* first_op, int32_t* widths, size_t capacity);

/* qsa_state_reset + a relabel of |0..0> to the plan's layout (metadata only,
 * valid for |0..0>, §IV-D) + qsa_plan_execute, without the reset's clearing
 * pass when the plan begins with a zero-state preparation (opts.zero_init,
 * N >= 12), which writes every amplitude.  The
 * state's previous contents and layout are discarded.  Errors: as
 * qsa_plan_execute. */
qsa_status qsa_plan_execute_from_zero(qsa_state s, qsa_plan p, qsa_run_stats* stats);

/* Execution order of the input ops (order[i] = input index of the i-th op
 * executed; the identity unless opts.layer moved ops); first_op of
 * qsa_plan_blocks indexes this order.  capacity >= n_ops, else QSA_E_RANGE. */
qsa_status qsa_plan_order(qsa_plan p, size_t* order, size_t capacity);

/* Kind of every block (0 dense, 1 diagonal, 2 product, 3 layer, 4 zero-state
 * preparation of the zero_init prefix) and, for
 * layer blocks, how many of its ops (the first ones in execution order) are
 * its diagonal part (0 for other kinds).  Nullable outputs; capacity >=
 * n_blocks, else QSA_E_RANGE. */
qsa_status qsa_plan_block_kinds(qsa_plan p, int32_t* kinds, int32_t* n_diag, size_t capacity);

/* Host-only replay of the promotions QSA_LOWER_PERMUTE makes for this plan
 * (§IV-D demand model; no data moves): starting from layout_in (host,
 * phys_of_logical, NULL = identity), each dense block's targets outside the
 * frames are promoted in target order, evicting per `victim` (qsa_victim);
 * diagonal blocks need no promotion.  *promotions = swapped position pairs,
 * *passes = blocks that promoted (one permutation pass each); layout_out
 * (host, N entries, nullable) receives the final layout.  Execution of the
 * plan with QSA_LOWER_PERMUTE and the same victim rule makes exactly these
 * promotions.  Errors: QSA_E_ARG (NULL plan, layout not a bijection, victim). */
qsa_status qsa_plan_promotions(qsa_plan p, const int32_t* layout_in, int victim, uint64_t* promotions,
                               uint64_t* passes, int32_t* layout_out);

/* A state sharded over 2^rank_bits ranks (§IV-D, Alg. lazy-mpi): the highest
 * rank_bits physical positions address the rank, rank R holding the slab of
 * 2^(N - rank_bits) amplitudes whose rank bits equal R.  A block whose
 * targets include a rank position needs that position swapped with a local
 * one first: one exchange step.  For the swap of rank position P with local
 * position l (j = P - (N - rank_bits)), rank R and its partner R ^ (1 << j)
 * exchange the halves of their slabs whose bit l differs from bit j of their
 * own rank index (2^(N - rank_bits - 1) amplitudes each way, written to the
 * same local slots); afterwards the layout holds the swap (the lazy
 * remapping of §IV-D, Eq. lazy-vol). */
typedef struct {
    uint64_t block;      /* the plan block the exchange precedes */
    int32_t rank_pos;    /* physical rank position (>= N - rank_bits) */
    int32_t local_pos;   /* physical local position (< N - rank_bits) it swaps with */
} qsa_exchange;

/* Host-only: the exchange steps of running plan p on 2^rank_bits ranks
 * (rank_bits in 1..N-1) from layout_in (host, phys_of_logical; NULL =
 * identity).  Every non-diagonal block (dense, product and layer blocks: the
 * qubits of their factors) has its targets made local before it runs, the
 * victim of each promotion chosen per `victim` (qsa_victim) among the local
 * positions not holding a target of the block; diagonal blocks need no
 * exchange (a rank knows its own rank bits).  Exchanges are listed in
 * execution order in out[0..capacity) (host; nullable when capacity is 0),
 * their count in *n_out; layout_out (host, N entries, nullable) receives the
 * final layout.  No data moves and no device is touched.  Errors: QSA_E_ARG
 * (NULL plan or n_out, rank_bits, layout, victim, a block wider than the
 * local positions), QSA_E_RANGE (capacity < *n_out; *n_out is set). */
qsa_status qsa_plan_exchanges(qsa_plan p, int rank_bits, const int32_t* layout_in, int victim, qsa_exchange* out,
                              size_t capacity, size_t* n_out, int32_t* layout_out);

/* Apply the plan's blocks to s in order (asynchronous unless opts.timing).
 * The first execution on a device uploads the fused matrices once
 * (stats->h2d_bytes).  Errors: QSA_E_ARG if the plan's N differs from s. */
qsa_status qsa_plan_execute(qsa_state s, qsa_plan p, qsa_run_stats* stats);

/* Free the plan (synchronises the device if matrices were uploaded). */
qsa_status qsa_plan_destroy(qsa_plan p);

/* Total kernels launched on this state since creation. */
qsa_status qsa_state_counters(qsa_state s, uint64_t* launches);

/* Wait for all work queued on the state's stream.  Returns QSA_E_TIMEOUT (and
 * marks the state failed) if a kernel's bounded wait gave up since the last
 * check, QSA_E_CUDA on a CUDA error.  Calls that return results to the host
 * make the same check. */
qsa_status qsa_state_sync(qsa_state s);

/* ---- outputs (§IV-E "Sampling", App. B "Numerical configuration") ----------- */

/* p_x = |psi_x|^2 in FP64 for every LOGICAL index x (decoded through L),
 * written to out_host (2^N doubles, may be NULL), and the FP64 norm
 * sum_x p_x to *norm_out (may be NULL).  Synchronises. */
qsa_status qsa_probabilities(qsa_state s, double* out_host, double* norm_out);

/* As qsa_probabilities but writes to a device buffer of 2^N doubles. */
qsa_status qsa_probabilities_device(qsa_state s, double* out_dev, double* norm_out);

/* <Z_mask> = sum_x (-1)^{popcount(x & logical_mask)} p_x (FP64 accumulation);
 * logical_mask = 0 gives the norm.  Synchronises. */
qsa_status qsa_expectation_z(qsa_state s, uint64_t logical_mask, double* out);

/* Several masks in one pass over the state (each result bit-identical to
 * qsa_expectation_z with that mask): logical_masks (host, n_masks entries,
 * each < 2^N), out (host, n_masks doubles).  Synchronises the stream.
 * Errors: QSA_E_ARG (n_masks outside 1..QSA_MAX_ZMASKS, a mask beyond N,
 * NULL). */
#define QSA_MAX_ZMASKS 4
qsa_status qsa_expectation_z_batch(qsa_state s, const uint64_t* logical_masks, int n_masks, double* out);

/* qsa_expectation_z for each of z_masks[0..n_masks) (logical, n_masks in
 * 0..QSA_MAX_ZMASKS) into z_out (host) and qsa_sample_counts (same draws and
 * outputs; §IV-E hierarchical sampling), the sums taken in the sampler's pass
 * over the state, so the state is read once for both (each sum agrees with qsa_expectation_z to FP64
 * rounding; the summation order differs).  Synchronises the stream.  Errors:
 * as qsa_sample_counts, and QSA_E_ARG for n_masks, a mask beyond N or NULL. */
qsa_status qsa_measure(qsa_state s, const uint64_t* z_masks, int n_masks, double* z_out, uint64_t shots,
                       uint64_t seed, uint64_t* outcomes, uint64_t* counts, size_t capacity, size_t* n_distinct);

/* Draw `shots` outcomes (§IV-E): integer weights
 * P_y = floor(re_y^2 * 2^60) + floor(im_y^2 * 2^60) of the stored FP32
 * amplitude (each square exact in FP64, so the weight is too; |amplitude| < 2
 * keeps it below 2^62), so the CDF does not depend on summation order, over
 * physical indices in
 * 2^10-amplitude blocks; shot i draws Philox4x64-10(ctr = (i, 0, 0, 0),
 *  key = (seed, 0)).word0 = r, maps it to u = floor(r * total / 2^64) and takes the first physical index whose
 * cumulative weight is strictly greater (a zero-weight bin is never drawn);
 * the outcome is decoded to the logical bitstring through L (§IV-D).
 * Results: distinct logical outcomes ascending in outcomes[], their counts in
 * counts[], *n_distinct.  If capacity < n_distinct: QSA_E_RANGE with
 * *n_distinct set and nothing written.  shots in 1..2^26.  Synchronises. */
qsa_status qsa_sample_counts(qsa_state s, uint64_t shots, uint64_t seed, uint64_t* outcomes, uint64_t* counts,
                             size_t capacity, size_t* n_distinct);

/* ---- batched trajectories ---------------------------------------------------
 * Many independent small states (noisy trajectories: the per-gate Pauli
 * channels of §IV-A sampled into explicit Pauli branches, so every trajectory
 * is a unitary circuit) evolved in ONE persistent kernel launch: each
 * thread-block cluster of four CTAs pops a trajectory from an atomic queue
 * (longest first), resets it to |0..0> and applies all of its fused blocks,
 * the four CTAs splitting every pass's tiles and meeting at a cluster barrier
 * between blocks; a second kernel samples every state (one CTA per
 * trajectory, Philox stream id = trajectory index, identity layout), and both
 * can be replayed as one captured CUDA graph. */
typedef struct qsa_batch_s* qsa_batch;

/* Host planning + one-time upload: trajectory t is ops[op_offsets[t] ..
 * op_offsets[t+1]) (op_offsets has n_traj + 1 entries, op_offsets[0] = 0).
 * N in 1..22; opts->kmax <= 4 (QSA_E_ARG otherwise). */
qsa_status qsa_batch_create(int n_qubits, int n_traj, const qsa_op* ops, const size_t* op_offsets,
                            const qsa_plan_opts* opts, qsa_batch* out);

/* Total fused blocks, input ops, and kernels launched so far. */
qsa_status qsa_batch_info(qsa_batch b, size_t* total_blocks, size_t* total_ops, uint64_t* launches);

/* Evolve every trajectory from |0..0> into dev_states (caller-owned device
 * buffer of >= n_traj * 8 * 2^N bytes, state t at offset t * 8 * 2^N) and
 * draw `shots` (1..16384) samples of each with the rule of qsa_sample_counts
 * (stream id t).  use_graph = 1 captures the launches into a CUDA graph on
 * first use (re-captured when an argument changes) and replays it.
 * budget_cycles > 0 bounds each cluster's run time in SM clock cycles (as seen
 * by its first CTA): a cluster that runs over stops between blocks and the
 * call returns QSA_E_TIMEOUT.
 * Synchronises cuda_stream; stats->seconds is the device time of the launch. */
qsa_status qsa_batch_run(qsa_batch b, void* dev_states, size_t bytes, uint64_t shots, uint64_t seed,
                         uint64_t budget_cycles, int use_graph, void* cuda_stream, qsa_run_stats* stats);

/* Copy the last run's samples to the host: for trajectory t, outcomes and
 * counts at [t * shots, t * shots + n_distinct[t]) (ascending outcomes). */
qsa_status qsa_batch_counts(qsa_batch b, uint32_t* outcomes, uint32_t* counts, uint32_t* n_distinct);

qsa_status qsa_batch_destroy(qsa_batch b);

/* ---- cost model: 37 -> 64 -> 64 -> 1 ReLU network on log-seconds ------------
 * Not in the paper (its planner score gamma "is not a runtime predictor",
 * §IV-C); it replaces gamma in Eq. dp-recurrence with predicted seconds.
 * Features x = [k/6, b_0..b_33 (physical target mask), N/34, log2(batch)/8].
 * Parameters: 6657 floats, W1[64][37], b1[64], W2[64][64], b2[64], W3[1][64],
 * b3[1], row-major.  All device pointers are caller-owned FP32 arrays. */
#define QSA_MLP_PARAMS 6657
#define QSA_MLP_FEATURES 37

/* Feature vector of a k-qubit pass on physical positions phys_mask (host out37). */
qsa_status qsa_costmodel_features(int k, uint64_t phys_mask, int n_qubits, int batch, float* out37);

/* Install (params != NULL, host, copied) or remove (NULL) the process-wide
 * model used by QSA_PLAN_DP_MLP. */
qsa_status qsa_costmodel_set(const float* params);

/* exp(f(x)) in seconds for n feature rows (host) with the installed model;
 * QSA_E_STATE if none is installed. */
qsa_status qsa_costmodel_predict(const float* features, size_t n, double* seconds_out);

/* Write the process-wide model to the file `path`: the 8 bytes "QSACM001",
 * the parameter count as a little-endian uint32 (6657), then the parameters
 * as little-endian float32 in the layout above.  Errors: QSA_E_STATE when no
 * model is installed, QSA_E_ARG when path is NULL or the file cannot be
 * written. */
qsa_status qsa_costmodel_save(const char* path);

/* Read a model file written by qsa_costmodel_save.  s == NULL installs it
 * process-wide (as qsa_costmodel_set); otherwise it is attached to s alone:
 * qsa_apply_circuit on s plans QSA_PLAN_DP_MLP with it, while other states,
 * qsa_plan_create and qsa_plan_circuit keep the process-wide model.  path ==
 * NULL detaches the state's model (s != NULL) or removes the process-wide one
 * (s == NULL).  The library keeps its own copy.  Errors: QSA_E_ARG for a file
 * that cannot be read, has the wrong header or count, trailing bytes, or a
 * non-finite parameter (nothing is changed then). */
qsa_status qsa_costmodel_load(qsa_state s, const char* path);

/* He-uniform initial parameters from a seed (host out). */
qsa_status qsa_costmodel_init(uint64_t seed, float* params_host);

/* Bytes of device workspace the MLP kernels need for n samples. */
size_t qsa_mlp_workspace_bytes(size_t n);

/* y_dev[s] = f(X_dev[s]) for s < n (X row-major n x 37).  Asynchronous. */
qsa_status qsa_mlp_forward(const float* params_dev, const float* X_dev, size_t n, float* y_dev, float* workspace_dev,
                           void* stream);

/* Loss L = mean_s (f(X_s) - t_s)^2 into *loss_dev (nullable) and dL/dparams
 * into grads_dev (6657 floats), by backpropagation.  Asynchronous. */
qsa_status qsa_mlp_loss_grad(const float* params_dev, const float* X_dev, const float* t_dev, size_t n,
                             float* grads_dev, float* loss_dev, float* workspace_dev, void* stream);

/* One Adam step (Kingma & Ba 2015) on count parameters, step number >= 1. */
qsa_status qsa_mlp_adam_step(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev, size_t count,
                             int step, float lr, float beta1, float beta2, float eps, void* stream);

/* Time one pass of n_samples random (k in 1..min(6,N), uniformly drawn
 * physical targets) fused operators on s (identity matrices: the amplitudes
 * are unchanged), median of reps launches each, at the given precision.
 * Fills X_host (n_samples x 37) and y_host (log seconds).  Synchronises. */
qsa_status qsa_costmodel_collect(qsa_state s, size_t n_samples, int reps, int precision, uint64_t seed,
                                 float* X_host, float* y_host);

/* Train on (X_host, y_host) with the library's GPU kernels: epochs of
 * shuffled minibatches, MSE loss on standardised targets (the mean and scale
 * are folded back into W3, b3) plus an L2 penalty (weight_decay/2)|p|^2,
 * Adam(lr, 0.9, 0.999, 1e-8).  The penalty keeps the network from fitting
 * noise through the 34 sparse mask features.  params_inout: initial
 * parameters in, trained parameters out (host).  epoch_loss_host (nullable,
 * epochs floats) receives the full-set MSE after each epoch. */
qsa_status qsa_costmodel_train(const float* X_host, const float* y_host, size_t n, int epochs, int batch, float lr,
                               float weight_decay, uint64_t seed, float* params_inout_host, float* epoch_loss_host);

/* Sampling that allocates nothing on the device.  The paper has no
 * counterpart: this exists for callers that cannot let the library call
 * cudaMalloc, e.g. a framework whose caching allocator owns the device memory
 * budget (at N = 33/34 the state fills most of HBM and a stray allocation can
 * fail or fragment the pool) or a pipeline that must not stall (cudaFree
 * synchronises the whole device).
 *
 * Same draws and results as qsa_sample_counts, but everything is caller-owned
 * except the scratch, which is one fixed device array of
 * QSA_NOALLOC_SCRATCH_WORDS 64-bit words (4 MiB) held by every GPU that loads
 * the library until the process exits.  Requests needing more scratch,
 * 2^max(N-10,0) + next_pow2(shots) + shots words (e.g. N <= 28 with 65536
 * shots), are rejected with QSA_E_RANGE before any launch.
 *   dev_amplitudes   device, 8*2^N bytes, 16-byte aligned, stored (physical) order;
 *   phys_of_logical  host, N entries, the layout map (a bijection);
 *   out_outcomes_dev, out_counts_dev  device, >= shots uint64 each: distinct
 *                    logical outcomes ascending and their counts;
 *   out_n_distinct_dev  device, one uint64.
 * Asynchronous on cuda_stream; nothing is copied to the host.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Every
 * call shares the one array, so calls that overlap on the GPU (other streams,
 * other threads) race; nothing in it needs clearing between calls.  An
 * all-zero state gives unspecified counts.  Errors: QSA_E_ARG, QSA_E_RANGE,
 * QSA_E_CUDA. */
#define QSA_NOALLOC_SCRATCH_WORDS (1u << 19)
qsa_status qsa_sample_counts_noalloc(const void* dev_amplitudes, int n_qubits, const int32_t* phys_of_logical,
                                     uint64_t shots, uint64_t seed, uint64_t* out_outcomes_dev,
                                     uint64_t* out_counts_dev, uint64_t* out_n_distinct_dev, void* cuda_stream);

/* ---- test hooks (host side) ------------------------------------------------
 * Failure injection without any device fault: the nth device allocation the
 * library makes from now on (0 = the next one) fails as if the device were
 * out of memory, so callers see QSA_E_NOMEM and the error paths release what
 * they had allocated; nth < 0 turns injection off.  The environment variable
 * QSA_FAULT_ALLOC=<n> sets the same when the library is loaded.  Not
 * thread-safe with respect to which allocation fails when several threads
 * allocate. */
qsa_status qsa_debug_fail_alloc(int64_t nth);

/* Device allocations the library currently holds (states it allocated, plan
 * and batch uploads, scratch): a leak check for the error paths. */
uint64_t qsa_debug_live_allocations(void);

/* Debug-build bounds checks.  A library built with -DQSA_DEBUG_BOUNDS
 * (paper_2608_16940_gb300/build.py --debug-bounds: libqsa_debug.so) checks the
 * state indices of the fused-update, permutation, product, batched, layer and
 * tensor-core kernels' global loads and stores; an out-of-range access is
 * skipped (no trap, no assert) and the first one of each kernel file is kept.
 * qsa_debug_bounds_status returns the first record found as
 * (check code << 48) | index, 0 when no check has failed (always 0 in a
 * release build); it reads device memory, so call it after the stream is
 * synchronised.  qsa_debug_bounds_enabled returns 1 in the debug build. */
uint64_t qsa_debug_bounds_status(void);
int qsa_debug_bounds_enabled(void);

const char* qsa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QSA_H */

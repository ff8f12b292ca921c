/*
 * zc.h -- C ABI of the ZeroCheck prover library (libzc.so).
 *
 * The library proves the ZeroCheck claim "f vanishes on the domain" in the
 * two forms compared by the paper "When Proofs Meet Hardware: Comparing NTT
 * and SumCheck in Zero-Knowledge Systems" (Fig. side-by-side-zc):
 *   - SumCheck form (multilinear ZeroCheck, Sec. 3.3, Eq. multilinear_zc_sc):
 *     sum_x f_M(x) eq_r(x) = 0 over {0,1}^n, proved in n Fiat-Shamir rounds;
 *   - NTT form (univariate ZeroCheck, Sec. 3.2): z_H | f, proved by the
 *     quotient q = f / z_H computed with INTT_H, a coset NTT over D, pointwise
 *     gate evaluation, division by z_H and INTT_D.
 * The field is the BLS12-381 scalar field
 *   r = 0x73eda753299d7d483339d80809a1d80553bda402fffe5bfeffffffff00000001.
 *
 * Data layout at the ABI.  A column is N = 2^n field elements, each 32 bytes,
 * the canonical integer in [0, r) as little-endian bytes, in natural order:
 * element i of a column is the value of the witness polynomial at the i-th
 * point of the domain (omega_N^i for the NTT form, the hypercube point whose
 * binary expansion is i, x_1 = most significant bit, for the SumCheck form).
 * Columns are passed as an array of c pointers.  Gates and column orders:
 *   ZC_GATE_PLONK   (d = 3, c = 8): [qL, qR, qM, qO, qC, a, b, c],
 *                   f = qL a + qR b + qM a b + qO c + qC;
 *   ZC_GATE_PRODUCT (d >= 2, c = d + 1): [q, w1, ..., w_{d-1}, o],
 *                   f = q w1 ... w_{d-1} - o;
 *   ZC_GATE_SUM_OF(m) (d >= 2, m >= 0, c = d + m <= 65): [g_1, ..., g_{d+m}],
 *                   f = g_1 ... g_d + g_{d+1} + ... + g_{d+m}: one product of
 *                   d columns plus m single columns, the family of
 *                   polynomials the paper evaluates (Sec. 5, Table
 *                   poly_examples: g1 g2 = ZC_GATE_SUM_OF(0) with d = 2,
 *                   g1 g2 + g3 + g4 + g5 = ZC_GATE_SUM_OF(3) with d = 2,
 *                   g1 g2 g3 g4 = ZC_GATE_SUM_OF(0) with d = 4).
 * The gate word is what the proof header and the transcript carry, so m is
 * bound into both.
 *
 * Ownership.  The caller owns every buffer it passes.  A context owns the
 * device scratch memory, constant tables and streams it creates, and reuses
 * them across calls; zc_destroy frees them.
 *
 * Errors.  No call throws; every call returns a zc_status.  On failure the
 * context keeps a message readable with zc_last_error.  A proof that does
 * not verify is reported as ZC_OK with *accept = 0; a malformed proof or
 * argument is ZC_ERR_ARG.  Column values >= r are rejected (ZC_ERR_ARG),
 * checked on the device.
 *
 * Threading.  Calls on one context are serialised by an internal mutex; use
 * one context per stream for concurrent proving.
 *
 * Proof byte formats (all integers little-endian):
 *   SumCheck: "ZCS1" | u32 gate | u32 n | u32 d | G_i(t) for i = 1..n,
 *             t = 0..d+1 | v_j = the columns' MLEs at alpha, j = 1..c.
 *             Size 16 + 32 (n (d + 2) + c).
 *   SumCheck, eq-factored (ZC_FORM_SUMCHECK_EQ): "ZCS2" | u32 gate | u32 n |
 *             u32 d | H_i(t) for i = 1..n, t = 0..d | v_j, j = 1..c.  Size
 *             16 + 32 (n (d + 1) + c).
 *   NTT:      "ZCN1" | u32 gate | u32 n | u32 d | u32 domain | root(q) |
 *             g_j(z), j = 1..c | q(z).  Size 20 + 32 + 32 (c + 1).  domain
 *             is log2 M, or log2 Mb | (log2 Ms + 1) << 8 for a step-radix
 *             domain of Mb + Ms points (see zc_params).
 * Transcript: S0 = SHA-256(tag | u32 form | u32 gate |
 * u32 n | u32 d | u32 domain (0 for SumCheck)); absorb(m): S = SHA-256(S|m);
 * squeeze: S = SHA-256(S | 0x43), challenge = int_le(S) mod r; tag is
 * "zerocheck-gb300/v1", or "zerocheck-gb300/v2" for ZC_FORM_SUMCHECK_EQ.  The column
 * and quotient commitments are stood in by root(v): a binary SHA-256 Merkle
 * tree over leaves of 64 canonical elements (the last leaf may be shorter;
 * at a level with an odd count the last node moves up unchanged),
 * root = SHA-256(u64 len | top).
 */
#ifndef ZC_H
#define ZC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ZC_OK = 0,
  ZC_ERR_ARG = 1,              /* bad argument, value >= r, malformed proof */
  ZC_ERR_OOM = 2,              /* device or host allocation failed / over budget */
  ZC_ERR_CUDA = 3,             /* a CUDA runtime call failed */
  ZC_ERR_TIMEOUT = 4,          /* a bounded device wait gave up */
  ZC_ERR_UNSUPPORTED = 5,      /* size or degree outside what the context was set up for */
  ZC_ERR_BUFFER_TOO_SMALL = 6  /* proof capacity below zc_proof_size */
} zc_status;

typedef enum { ZC_GATE_PLONK = 1, ZC_GATE_PRODUCT = 2, ZC_GATE_SUM = 3 } zc_gate;
/* Gate word of the sum gate with m single columns (m in bits 8..15). */
#define ZC_GATE_SUM_OF(m) ((uint32_t)ZC_GATE_SUM | ((uint32_t)(m) << 8))
/* ZC_FORM_SUMCHECK_EQ: the SumCheck form with eq-factored round messages
 * (see zc_prove_sumcheck_eq). */
typedef enum { ZC_FORM_SUMCHECK = 1, ZC_FORM_NTT = 2, ZC_FORM_SUMCHECK_EQ = 3 } zc_form;

/* One ZeroCheck instance: gate word, n (N = 2^n, 1 <= n <= 28), degree d
 * (3 for Plonk, 2..64 for the product and sum gates) and the NTT form's
 * domain word log_blowup (SumCheck ignores it):
 *   - 0: |D| = next_pow2(d) N, the coset 7 <w_|D|>;
 *   - k (1..): |D| = 2^k N, the coset 7 <w_{2^k N}>;
 *   - ZC_DOMAIN_STEP(k, s), s < k: the step-radix domain of 2^k N + 2^s N
 *     points, 7 <w_{2^k N}> u sigma <w_{2^s N}> with sigma = 7 w_{2^{k+1} N}
 *     (Sec. 4, "Degree scaling": a non-power-of-two transform such as
 *     3N = 2N + N built from power-of-two transforms plus element-wise work).
 *     The library proves s = 0 (2^k N + N: 3N, 5N, 9N, ...).
 * |D| must hold the quotient's (d-1)N - d + 1 coefficients (Sec. 4 sizes the
 * quotient transform by the degree of q: 2N for degree 3, 3N for degree 4).
 * The NTT proof header and transcript carry log2 |D|, or for a step-radix
 * domain log2(2^k N) | (log2(2^s N) + 1) << 8; q has |D| coefficients. */
#define ZC_DOMAIN_STEP(k, s) ((uint32_t)(k) | (((uint32_t)(s) + 1u) << 8))
typedef struct {
  uint32_t gate, n, d;
  uint32_t log_blowup;
} zc_params;

/* device: CUDA ordinal.  max_n / max_d: largest instance the context will
 * accept (scratch grows on demand up to mem_budget_bytes; 0 = no budget). */
typedef struct {
  int device;
  uint32_t max_n, max_d;
  uint64_t mem_budget_bytes;
} zc_setup_opts;

typedef struct zc_ctx zc_ctx;

/* Create a context on opts->device: field and twiddle constants, streams.
 * Returns ZC_ERR_ARG for a null pointer, ZC_ERR_CUDA if the device cannot be
 * used.  Paper: the set-up the hardware designs of Sec. 4 assume (twiddle
 * buffers, Build-MLE unit). */
zc_status zc_setup(const zc_setup_opts* opts, zc_ctx** out);

/* Free everything the context owns.  Null is ignored. */
void zc_destroy(zc_ctx* ctx);

/* Proof size in bytes for params and form (formats above). */
zc_status zc_proof_size(const zc_params* params, zc_form form, size_t* bytes);

/* SumCheck-form ZeroCheck proof (Fig. side-by-side-zc right; Sec. 3.3).
 * cols: c pointers to N*32-byte canonical columns, device pointers when
 * cols_on_device != 0, host pointers otherwise (copied to the device inside
 * the call; from n = 18 on, with col_roots given, in eight pair ranges on the
 * context's copy stream while round 1 runs on the ranges already copied, so
 * pinned host memory lets the copy overlap the proof).  col_roots: the c column commitments root(col_j) if the caller
 * has them (stage (1) of the prover workflow, Sec. 3.1), or NULL to compute
 * them on the device.  cuda_stream: a cudaStream_t (NULL = legacy default).
 * proof: cap bytes, host or device memory; *len receives the proof size.
 * With device columns and a device proof buffer the call is asynchronous on
 * cuda_stream; otherwise it returns after the proof is written. */
zc_status zc_prove_sumcheck(zc_ctx* ctx, const zc_params* params, const void* const* cols,
                            int cols_on_device, const uint8_t (*col_roots)[32],
                            void* cuda_stream, uint8_t* proof, size_t cap, size_t* len);

/* SumCheck-form proof with eq-factored round messages (Sec. 3.3 with the
 * eq factor split off, the faster-prover formulation the paper cites with
 * Build MLE): round i's polynomial is G_i(X) = c_i l_i(X) H_i(X), with
 * c_i = prod_{j<i} eq(alpha_j, r_j) and l_i(X) = (1 - r_i)(1 - X) + r_i X
 * known to the verifier, so the round sends H_i (degree d) at X = 0..d:
 * d + 1 values instead of G_i's d + 2, and one SHA-256 block less per
 * round for low degrees.  The verifier checks c_i ((1 - r_i) H_i(0) +
 * r_i H_i(1)) against the claim.  Proof format "ZCS2" (above), transcript
 * tag v2 with form word ZC_FORM_SUMCHECK_EQ.  Arguments, asynchrony and
 * errors as for zc_prove_sumcheck. */
zc_status zc_prove_sumcheck_eq(zc_ctx* ctx, const zc_params* params, const void* const* cols,
                               int cols_on_device, const uint8_t (*col_roots)[32],
                               void* cuda_stream, uint8_t* proof, size_t cap, size_t* len);

/* NTT-form ZeroCheck proof (Fig. side-by-side-zc left; Sec. 3.2).
 * Arguments as for zc_prove_sumcheck.  q_out: NULL, or M*32 bytes
 * (M = |D| points of the domain, see zc_params) that receive the quotient coefficients q_0..q_{M-1},
 * canonical, device memory when q_on_device != 0 (M = |D|, see zc_params).
 * Asynchronous when the columns, proof and q_out are all device memory. */
zc_status zc_prove_ntt(zc_ctx* ctx, const zc_params* params, const void* const* cols,
                       int cols_on_device, const uint8_t (*col_roots)[32], void* cuda_stream,
                       uint8_t* proof, size_t cap, size_t* len, void* q_out, int q_on_device);

/* Verify a proof on the host (no device needed).  cols: host columns (oracle
 * access in place of a commitment opening).  q: the quotient (NTT form,
 * M*32 bytes host memory; ignored for SumCheck).  *accept = 1 iff every
 * check passes: per-round G_i(0)+G_i(1) = G_{i-1}(alpha_{i-1}) (Sec. 3.4),
 * the final eq-weighted gate check and v_j = MLE_j(alpha) (Sec. 3.3); or
 * root(q), deg q <= deg f - N, q(z), the openings g_j(z) and
 * gate(g(z)) = z_H(z) q(z) (Sec. 3.2).  Malformed input: ZC_ERR_ARG. */
zc_status zc_verify(const zc_params* params, zc_form form, const void* const* cols,
                    const uint8_t (*col_roots)[32], const uint8_t* proof, size_t len,
                    const void* q, int* accept);

/* Column commitments root(col_j) for j < c, computed on the device
 * (Fig. side-by-side-zc, "Commit"; stand-in described above).  roots_out:
 * host memory, c entries.  Synchronous. */
zc_status zc_roots(zc_ctx* ctx, const zc_params* params, const void* const* cols,
                   int cols_on_device, void* cuda_stream, uint8_t (*roots_out)[32]);

/* Device-side timing of the last prove call on ctx, from CUDA events the
 * library records on the call's stream.  Writes min(cap, 10) values:
 * [0..5] phase times in ms.  SumCheck: roots, transcript r + eq tables,
 * round-1 evaluation kernel, rounds 2..n, final values + proof out.  NTT:
 * roots, INTT_H, slice LDE + gate + divide, q INTT, q root + z, openings +
 * proof out.  [6] time of the dominant kernel launch (ms), [7] its
 * algorithmic modular multiplications, [8] its algorithmic DRAM bytes,
 * [9] number of kernels the call launched.  Waits for the call's events. */
zc_status zc_stats(zc_ctx* ctx, double* phase_ms, uint32_t cap);

/* ---- Batched proving (deployment mode; the paper proves one instance at a
 * time).  A batch of `count` instances, each with its own form, params and
 * DEVICE columns, DEVICE proof buffer (zc_proof_size bytes) and, for the NTT
 * form, an optional DEVICE q buffer (NULL entries allowed).  The context
 * runs the batch on up to 16 lanes (concurrent streams with their own
 * scratch), longest instance first onto the least-loaded lane; every proof
 * is byte-identical to the one zc_prove_sumcheck / zc_prove_ntt returns for
 * the same instance.  Column roots are computed on the device. */

/* Prove a batch now, asynchronously on cuda_stream (scratch is allocated
 * before the kernels are queued, which may synchronise the device). */
zc_status zc_prove_batch(zc_ctx* ctx, uint32_t count, const zc_form* forms, const zc_params* params,
                         const void* const* const* cols, void* cuda_stream, uint8_t* const* proofs,
                         void* const* q_outs);

typedef struct zc_batch zc_batch;

/* Allocate everything a batch needs, then capture its whole launch sequence
 * into one CUDA graph.  The graph keeps the given pointers: relaunching it
 * proves whatever the column buffers hold at launch time. */
zc_status zc_batch_create(zc_ctx* ctx, uint32_t count, const zc_form* forms, const zc_params* params,
                          const void* const* const* cols, uint8_t* const* proofs, void* const* q_outs,
                          zc_batch** out);

/* One graph launch proves every instance of the batch (asynchronous). */
zc_status zc_batch_launch(zc_batch* batch, void* cuda_stream);

/* Kernels the batch graph contains. */
uint32_t zc_batch_kernels(const zc_batch* batch);

/* Free the graph (the context keeps its lanes for later batches). */
void zc_batch_destroy(zc_batch* batch);

/* SumCheck-form proof without any device allocation (the paper has no
 * counterpart; this is a deployment variant of zc_prove_sumcheck).
 *
 * For callers that cannot allocate device memory while proving: code whose
 * memory is handed out by an external pool reserved up front, pipelines
 * that must not incur the implicit device synchronisation of
 * cudaMalloc/cudaFree, or processes whose device memory is already fully
 * reserved.  All scratch memory lives in fixed-size file-scope device arrays
 * of the library (32 MiB of scratch plus constant tables, held by every GPU
 * that loads the library until the process exits).  No context is used and
 * nothing is allocated: no cudaMalloc, cudaFree or allocating routine.
 *
 * params: as for zc_prove_sumcheck.  cols: c DEVICE pointers (N*32 canonical
 * bytes each) on the current device.  col_roots: host array of c roots, or
 * NULL to compute them inside the static scratch; given roots are copied
 * from the caller's (pageable) host array by a host-to-device copy queued on
 * cuda_stream, which a stream capture cannot record: under capture pass
 * col_roots = NULL.  cuda_stream: the stream the work is queued on.  proof:
 * DEVICE buffer of cap bytes; *len receives the proof size.  The call is
 * asynchronous: the proof is ready when the stream reaches it.  The bytes
 * equal zc_prove_sumcheck's.
 *
 * Errors: argument and size errors are returned at once.  A column value
 * >= r cannot be reported by the return status, because the call does not
 * wait for the device: the proof buffer then starts with the four bytes
 * "ZCE!" instead of "ZCS1", and the caller checks them once the stream has
 * completed (zc_prove_sumcheck returns ZC_ERR_ARG for the same input).
 *
 * Limits: the instance must fit the 32 MiB scratch (tables c*N*32 bytes plus
 * small per-round buffers, e.g. the Plonk gate up to n = 16; with
 * col_roots = NULL also the commitment's node buffers); larger instances
 * return ZC_ERR_UNSUPPORTED without launching anything.  The environment
 * variable ZC_STATIC_SCRATCH_BYTES, if set, lowers the usable part of the
 * scratch (for tests of the size checks).
 * Set-up: the first call on each device looks up the device addresses of the
 * static arrays (cudaGetSymbolAddress) with that device current and copies
 * the field constants into them with synchronous copies, so make that first
 * call outside any stream capture.  The set-up is redone when the device's
 * CUDA context changes (after cudaDeviceReset the arrays are new), so the
 * first call after such a reset is a set-up call too.  Sharing: every call on a device uses the
 * same arrays and leaves its data in them (the per-proof state is reset by
 * the call itself), so calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and corrupt each other; order
 * them on one stream. */
zc_status zc_prove_sumcheck_static(const zc_params* params, const void* const* cols,
                                   const uint8_t (*col_roots)[32], void* cuda_stream,
                                   uint8_t* proof, size_t cap, size_t* len);

/* ------------------------------------------ commitment around it --
 * Stages (1) and (3) of the prover workflow (Sec. 3.1) around the ZeroCheck,
 * with the lightweight hash-based commitment the paper points to (Ligero):
 * commit to the c witness columns before proving, then open them at the
 * point alpha the SumCheck form ends in, so that a verifier checks the
 * proof's final values v_j against the commitment instead of reading the
 * columns.  Layout: each column (an MLE table of N = 2^n values, x_1 the
 * most significant index bit) is an m x w matrix, w = 2^nc, m = N / w.
 * Commit: every row is Reed-Solomon encoded at rate 1/4 (the values of the
 * row polynomial at the W = 4w points 7 w_W^k); leaf k = SHA-256 of the
 * SHA-256 digests of position k of each encoded column (its m entries);
 * root = SHA-256(u64 W | top of the binary Merkle tree of the W leaves).
 * Open: u_j = sum_i eq(alpha_1..nr, i) row_i of column j, a random
 * combination u' of all rows (proximity test), and t queried positions with
 * their encoded columns and Merkle paths; transcript SHA-256(
 * "zerocheck-gb300/pcs-v1" | u32 n | u32 nc | u32 c | u32 t | root |
 * enc(alpha_i) | enc(v_j)), absorb/squeeze as above, query k = low 64 bits
 * of a challenge mod W.  Proof "ZCP1" | u32 n | u32 nc | u32 c | u32 t |
 * u_j | u' | per query: the c m entries, then log2 W sibling digests from
 * the leaf up.  With the ZeroCheck, the caller passes the PCS root as every
 * column's root (col_roots[j] = root), which binds the commitment into the
 * ZeroCheck transcript.  Soundness of a query set: each query catches a
 * matrix far from the code with probability >= 3/8 (t = 189 for 2^-128). */
typedef struct {
  uint32_t n;   /* columns of 2^n values, 1 <= n <= 24 */
  uint32_t nc;  /* rows of 2^nc values, 1 <= nc <= min(n, 12); 0: min(n, 12) */
  uint32_t c;   /* columns, 1..65 */
  uint32_t t;   /* queried positions of an opening, >= 1 */
} zc_pcs_params;

typedef struct zc_pcs zc_pcs;

/* Opening proof size: 20 + 32 (c w + w + t c m + t (nc + 2)). */
zc_status zc_pcs_proof_size(const zc_pcs_params* params, size_t* bytes);

/* Encode and commit to the c columns (host or device, canonical).  The
 * handle keeps the encoded columns (4 c N 32 bytes of device memory) and,
 * for device columns, the caller's pointers, whose contents must not change
 * until the handle is destroyed.  root: 32 bytes out.  Synchronous. */
zc_status zc_pcs_commit(zc_ctx* ctx, const zc_pcs_params* params, const void* const* cols,
                        int cols_on_device, void* cuda_stream, zc_pcs** out, uint8_t root[32]);

/* Opening of every column at alpha (n canonical elements) with the claimed
 * values (c canonical elements).  proof: host memory of cap bytes, *len the
 * size.  Synchronous. */
zc_status zc_pcs_open(zc_pcs* pcs, const uint8_t (*alpha)[32], const uint8_t (*values)[32],
                      void* cuda_stream, uint8_t* proof, size_t cap, size_t* len);

/* Host verifier of an opening against root: *accept = 1 iff every check
 * passes; ZC_ERR_ARG for a malformed proof. */
zc_status zc_pcs_verify(const zc_pcs_params* params, const uint8_t root[32], const uint8_t (*alpha)[32],
                        const uint8_t (*values)[32], const uint8_t* proof, size_t len, int* accept);

void zc_pcs_destroy(zc_pcs* pcs);

/* The point a SumCheck-form proof ends in: replays its transcript with the
 * given column roots (host, no columns needed) and writes alpha (n
 * canonical elements) and the proof's final values (c elements); *rounds_ok
 * = 1 iff every round's check and the final check gate(v) eq(r, alpha) =
 * claim pass (Sec. 3.3, 3.4).  With zc_pcs_verify on (alpha, values) this
 * verifies a ZeroCheck without the columns.  form: ZC_FORM_SUMCHECK or
 * ZC_FORM_SUMCHECK_EQ. */
zc_status zc_sumcheck_point(const zc_params* params, zc_form form, const uint8_t (*col_roots)[32],
                            const uint8_t* proof, size_t len, uint8_t (*alpha_out)[32],
                            uint8_t (*values_out)[32], int* rounds_ok);

/* ----------------------------------------------------------- serving --
 * A request loop over a list of timed requests (the paper proves one
 * instance at a time; serving is a deployment mode of the same arithmetic).
 * Requests become visible at their arrival time; each is admitted when a
 * slot (a stream with its own child context) is free AND its scratch fits in
 * a device pool of hbm_budget_bytes (first fit).  Admitted proofs run
 * concurrently; their tables and transcripts live in the pool block until
 * completion is observed, when the block and slot return for the next
 * admission (continuous batching).  Every proof is byte-identical to the one
 * zc_prove_sumcheck / zc_prove_ntt returns for the same request.
 *
 * Scratch bytes one proof takes (device columns, roots computed on the
 * device; q_on_device: the NTT quotient goes to a caller buffer). */
zc_status zc_scratch_bytes(zc_ctx* ctx, const zc_params* params, zc_form form, int q_on_device,
                           size_t* bytes);

typedef struct {
  double arrival_s;           /* seconds after the run starts */
  zc_params params;
  zc_form form;               /* the form chosen for this request (a router's job) */
  const void* const* cols;    /* DEVICE columns, canonical (read only; may be shared) */
  uint8_t* proof;             /* DEVICE buffer of zc_proof_size bytes */
  void* q_out;                /* NTT form: DEVICE buffer of M*32 bytes, or NULL */
} zc_request;

typedef struct {
  double admit_s;             /* when it got its slot and scratch (run clock) */
  double done_s;              /* when its completion was observed (run clock) */
  uint64_t scratch_bytes;     /* the footprint it was admitted with */
  uint32_t slot;
  uint32_t waited_for_memory; /* 1 if a free slot waited for pool space for it */
  zc_status status;
} zc_result;

typedef struct {
  uint32_t slots;             /* proofs in flight at most, 1..64 */
  uint64_t hbm_budget_bytes;  /* size of the scratch pool (allocated once, kept) */
  uint32_t in_order;          /* 1: admit strictly by arrival; 0: a request that
                                 does not fit yet lets later ones that fit pass */
  double timeout_s;           /* ZC_ERR_TIMEOUT if the run lasts longer (0: none) */
  uint64_t priority_bytes;    /* 0: every slot alike.  Otherwise requests whose
                                 scratch is at least this many bytes run on slot 0,
                                 a stream of the device's greatest priority, one at
                                 a time in arrival order, and smaller requests use
                                 the other slots around them */
} zc_serve_opts;

/* Run the loop until every request completed; results[i] for reqs[i].
 * Blocks the calling thread (host clock: steady, seconds).  A request whose
 * scratch exceeds the whole pool fails alone with ZC_ERR_OOM in its result.
 * Returns the first failure status (results are filled in either case). */
zc_status zc_serve(zc_ctx* ctx, const zc_request* reqs, uint32_t count, const zc_serve_opts* opts,
                   zc_result* results);

/* ------------------------------------------------------------ tuning --
 * Launch parameters of the kernels, per form and size.  The paper fixes the
 * arithmetic, not the launch shape; every value gives byte-identical proofs
 * and only changes speed.  A tuner (paper_2606_16146_gb300/tune.py) measures
 * the candidates and stores the winners here.
 *
 *   ZC_TUNE_SC_GRID      SumCheck: most CTAs one round kernel is split over
 *                        (the fold/evaluate split); 1..4096, default one wave
 *                        of resident CTAs (Plonk) or two (product gate).
 *   ZC_TUNE_SC_TAIL_LOG  SumCheck: the single-CTA tail takes over once a round
 *                        has at most 2^value pairs (the Plonk tail starts at
 *                        round 2 at the earliest); 1..24, default 5.
 *   ZC_TUNE_SC_SMALL_LOG SumCheck: rounds 2.. with at most 2^value pairs
 *                        evaluate both H(0) and H(1) instead of deriving one
 *                        from the claim; 1..24, default 14.
 *   ZC_TUNE_SC_CHUNK_LOG SumCheck, Plonk gate: rounds 2.. with at most 2^value
 *                        pairs spread each pair over 16 threads; 1..24,
 *                        default 14.  From n = 20 on, the rounds inside the
 *                        cooperative round kernel take 16 threads per pair
 *                        when they evaluate both H(0) and H(1)
 *                        (ZC_TUNE_SC_SMALL_LOG) and 4 otherwise.
 *   ZC_TUNE_SC_MINB      SumCheck, Plonk gate: resident CTAs per SM the large
 *                        round kernels are compiled for; 1 or 2, default 2.
 *   ZC_TUNE_SC_PROD_PPT  SumCheck, product gate: evaluation points per thread
 *                        in the large rounds; 1 or 3, default per round (3 for
 *                        at most 3 points, 1 for 4-5 points or at most 2^16
 *                        pairs, else 3).
 *   ZC_TUNE_SC_QUAD_LOG  SumCheck, Plonk gate: rounds 2.. above the chunk
 *                        threshold with at most 2^value pairs spread each pair
 *                        over 4 threads (larger rounds: one pair per thread);
 *                        from n = 20 on they run inside the cooperative round
 *                        kernel; 1..24, default 17.
 *   ZC_TUNE_SC_PROD_FUSE SumCheck, product gate: rounds 2.. with at most
 *                        2^value pairs fold inside the evaluation kernel
 *                        (larger rounds: a separate MLE-update kernel);
 *                        1..24, default 16.
 *   ZC_TUNE_BATCH_LANES  batches: concurrent lanes (streams); set with n = 0
 *                        under either form; 1..64, default 16.
 *   ZC_TUNE_NTT_TILE_LOG NTT: elements per shared-memory pass tile, 2^value;
 *                        10, 11 or 12, default 11.
 *   ZC_TUNE_NTT_TWO_LOG  NTT: sizes 2^n with n >= value run each transform as
 *                        two four-step passes (more, smaller CTAs), smaller
 *                        ones as one pass (always two above n = 12); 2..24,
 *                        default 12.
 *   ZC_TUNE_NTT_MINB     NTT: resident CTAs per SM the 2^11 tile is compiled
 *                        for; 1 or 2, default 2.
 *
 * n = 0 sets the value for every size without its own entry; value = 0
 * removes an entry.  Out-of-range keys, forms, sizes or values give
 * ZC_ERR_ARG. */
typedef enum {
  ZC_TUNE_SC_GRID = 1,
  ZC_TUNE_SC_TAIL_LOG = 2,
  ZC_TUNE_NTT_TILE_LOG = 3,
  ZC_TUNE_NTT_MINB = 4,
  ZC_TUNE_SC_SMALL_LOG = 5,
  ZC_TUNE_SC_MINB = 6,
  ZC_TUNE_SC_PROD_PPT = 7,
  ZC_TUNE_SC_CHUNK_LOG = 8,
  ZC_TUNE_BATCH_LANES = 9,
  ZC_TUNE_SC_QUAD_LOG = 10,
  ZC_TUNE_SC_PROD_FUSE = 11,
  ZC_TUNE_NTT_TWO_LOG = 12
} zc_tune_key;

zc_status zc_tune_set(zc_ctx* ctx, zc_form form, uint32_t n, zc_tune_key key, int32_t value);

/* The value proofs of (form, n) use for key (the default when none is set). */
zc_status zc_tune_get(zc_ctx* ctx, zc_form form, uint32_t n, zc_tune_key key, int32_t* value);

/* Message describing the last failure on ctx ("" if none). */
const char* zc_last_error(zc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ZC_H */

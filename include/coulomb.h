/*
 * coulomb.h -- C ABI of the compressed Coulomb-integral engine for planewave bases
 * (Pederson, "Practical and Rigorous Reduction of the Many-Electron Quantum Mechanical
 * Coulomb Problem to O(N^{2/3}) Storage", arXiv:1502.08043).
 *
 * The Coulomb kernel is factorised through a Laplace transform (Sec. II, Eqs. 3-7), the
 * change of variable t = alpha^{-1/2} for the infinite interval (Eq. 11) and Gauss
 * quadrature (Eqs. 12-14) into S one-dimensional tables T_s[Delta] with weights w_s, so
 * that every two-electron integral is rebuilt from O(N^{2/3}) numbers (Sec. III).
 *
 * Conventions shared by every entry point
 *  - Units: Hartree atomic units; box side L in bohr.
 *  - Basis: integer vectors n with |n|^2 <= R^2 (planewaves exp(i 2 pi n.r / L)),
 *    lexicographic (n_x, n_y, n_z) order; the id of a function is its rank.
 *  - Integrals are chemists' (IJ|KL) with complex conjugates on I and K:
 *    nonzero only if n_J - n_I + n_L - n_K = 0, then V(q), q = n_J - n_I.
 *  - Kernels: CC_KERNEL_PERIODIC, V(q) = 4 pi / (Omega |q|^2) = 1/(pi L |n|^2), with the
 *    q = 0 term excluded (returned as 0).  CC_KERNEL_BOX, the free-space Coulomb kernel
 *    inside a finite box of side L (the model of the paper's Table I); q = 0 included.
 *  - Memory: every pointer named *_dev is device memory owned by the caller; *_host is
 *    host memory owned by the caller.  Tables are owned by the library behind the
 *    opaque handle.  No hot call (reconstruct, pair matrix, exchange) allocates.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Hot calls are asynchronous and stream ordered; argument errors are
 *    returned synchronously before anything is enqueued.  Build, info, save, load and
 *    free synchronise.
 *  - Errors: every function returns a cc_status; no C++ exception crosses the ABI, no
 *    device trap or assert is used.  Data-dependent problems found on the device
 *    (out-of-range ids) are counted in caller-provided counters, never fatal.
 *  - Threading: a handle is immutable after build and may be used from several host
 *    threads at once for different calls on different streams, except that two calls
 *    of cc_exchange_sums on one handle share its workspace and must be stream ordered.
 */
#ifndef COULOMB_H_
#define COULOMB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CC_OK = 0,
  CC_ERR_ARG = 1,      /* invalid argument (NULL pointer, size, enum) */
  CC_ERR_RANGE = 2,    /* size beyond a documented limit */
  CC_ERR_CUDA = 3,     /* a CUDA runtime call failed (message: cc_last_error) */
  CC_ERR_ALLOC = 4,    /* device or host allocation failed */
  CC_ERR_TIMEOUT = 5,  /* a bounded device wait ran out */
  CC_ERR_NOTSUPP = 6,  /* valid but unsupported combination */
  CC_ERR_IO = 7        /* file read/write or format error */
} cc_status;

typedef enum { CC_KERNEL_PERIODIC = 0, CC_KERNEL_BOX = 1 } cc_kernel;

typedef enum {
  CC_PREC_FP64 = 0,    /* double tables, double outputs */
  CC_PREC_FP32 = 1,    /* float tables, float outputs (plain FP32 path) */
  CC_PREC_BF16X3 = 2,  /* exchange only: bf16 hi+lo split operands on tensor cores */
  CC_PREC_FP16X3 = 3   /* exchange only: fp16 hi+lo split with per-node exponent scaling */
} cc_precision;

typedef enum {
  CC_LOOKUP_SEPARABLE = 0, /* Eq. 14 node sum: sum_s w_s T_s[q_x] T_s[q_y] T_s[q_z] */
  CC_LOOKUP_COLLAPSED = 1, /* periodic only: one table over m = |q|^2 (node sum folded) */
  CC_LOOKUP_GENERAL = 2    /* box only: any quadruple, conserving or not, from the
                              two-index per-axis tables A(alpha_s, D1, D2) of Eq. 8 */
} cc_lookup;

typedef enum {
  CC_QUAD_IDS_I32 = 0, /* int32[n][4] basis ids (I, J, K, L), 16 B per quadruple */
  CC_QUAD_VEC_I8X4 = 1, /* int8[n][4][4]: the four vectors (n_x, n_y, n_z, unused), 16 B */
  CC_QUAD_IDS_U16 = 2  /* uint16[n][4] basis ids, 8 B per quadruple; basis <= 65536 */
} cc_quad_format;

/* Quadrature and table parameters (Sec. II Eqs. 11-14 and the Table I meshes).
 *   kernel    cc_kernel.
 *   R         basis cutoff |n|^2 <= R^2, 1 <= R <= 127.  Tables cover Delta = 0..2R.
 *   L         box side (bohr), > 0.
 *   S         total number of quadrature nodes, 2 <= S <= 1024.
 *   n_sub     interval [0, alpha_c] is split at alpha_c ratio^-n_sub, ..., alpha_c/ratio
 *             (n_sub + 1 Gauss-Legendre sub-intervals; 0 = one interval, the paper's
 *             Mesh 1; 7 with ratio 5 = the paper's Mesh 2).  < 0 selects the default rule.
 *   q_tail    Gauss-Legendre points in t = alpha^{-1/2} on (0, alpha_c^{-1/2}] (Eq. 11);
 *             < 0 selects the default rule.
 *   alpha_c   split point (Sec. II fixes alpha_c = 1).  PERIODIC: in index units
 *             a = alpha (2 pi / L)^2; BOX: in bohr^2.  <= 0 selects 1.
 *   prune_tol PERIODIC only: drop node s when w_s exp(-a_s) < prune_tol / (12 R^2);
 *             0 keeps all nodes.  Negative selects 1e-9.  Ignored for BOX.
 *   ratio     sub-interval ratio of the split of [0, alpha_c] (the paper's Mesh 2: 5);
 *             <= 1 selects 5.
 * Default rule: (S, R) = (32, 4) -> (2, 10); (64, 13) -> (3, 21); (96, 31) -> (4, 29);
 * (128, 63) -> (5, 34); otherwise a search: with r = max(1, floor(log5(12 R^2)) - 1),
 * n_sub in {r, r + 1} and q_tail in 3 .. max(3, round(0.45 S)) (S - q_tail >= n_sub + 1),
 * the pair minimising max_m |sum_s w_s exp(-a_s m) - 1/m| m over the 96 points
 * m_k = 1 + floor((12 R^2 - 1) k^3 / 95^3), floored at 1e-10 (ties within 0.1 % go to the smaller
 * n_sub, then q_tail); fewer than 5 nodes: (0, S / 2).  The same rule applies to BOX
 * tables (give the paper's meshes explicitly there).  Every sub-interval gets
 * floor((S - q_tail)/(n_sub + 1)) points and the first (S - q_tail) mod (n_sub + 1)
 * get one more. */
typedef struct {
  int kernel;
  int R;
  double L;
  int S;
  int n_sub;
  int q_tail;
  double alpha_c;
  double prune_tol;
  double ratio;
} cc_table_params;

typedef struct cc_tables_s* cc_tables;

typedef struct {
  int kernel, R, S, n_sub, q_tail;
  double L, alpha_c, prune_tol;
  int S_eff;          /* nodes kept after pruning */
  int Nb;             /* basis size */
  int Mg;             /* grid side 2R + 1 */
  int m_max;          /* collapsed table covers m = 0..m_max = 4 R^2 */
  size_t device_bytes; /* device memory held by the handle (tables + workspace) */
  size_t table_bytes;  /* of which the FP32 lookup tables (the stored compression) */
  double ratio;        /* sub-interval ratio of the mesh */
  int general_codes;   /* BOX: entries per node of the two-index tables, (2R + 1)^2; 0 for
                          PERIODIC (Sec. III counts 4 N^{2/3} per node for N planewaves) */
  size_t general_table_bytes; /* BOX: FP32 two-index lookup tables, general_codes x S_eff
                                 entries padded to S_eff rounded up to 32; 0 for PERIODIC */
} cc_tables_info_t;

/* Build the node set, weights and tables on the device of the current context
 * (Sec. II Eqs. 11-14; nodes, weights and table entries in FP64 on the GPU).  Also
 * allocates the exchange workspace of this cutoff.  Synchronous.
 * Errors: CC_ERR_ARG / CC_ERR_RANGE for bad parameters, CC_ERR_ALLOC, CC_ERR_CUDA. */
cc_status cc_build_tables(const cc_table_params* params, void* stream, cc_tables* out);

/* Sizes and resolved parameters of a handle. */
cc_status cc_tables_info(cc_tables t, cc_tables_info_t* info);

/* Copy the full node set (before pruning) to the host: alpha[S], w[S] (Laplace
 * variable of the kernel's units and Eq. 14 weights), part[S] (0: [0, alpha_c],
 * 1: tail), kept[S] (1 if the node survives pruning).  Any pointer may be NULL. */
cc_status cc_tables_nodes(cc_tables t, double* alpha_host, double* w_host, int* part_host,
                          int* kept_host);

/* Copy the FP64 per-node tables of the kept nodes to the host:
 * table_host[S_eff][2R + 1] = T_s[Delta] (PERIODIC exp(-a_s Delta^2), BOX A(alpha_s, Delta)). */
cc_status cc_tables_values(cc_tables t, double* table_host);

/* BOX tables only: copy the FP64 two-index per-axis tables of the kept nodes to the host,
 * table_host[S_eff][(2R + 1)^2] = A(alpha_s, d1, d2) (Sec. II Eq. 8 with box-normalised
 * planewaves on [0, L]: A = 1/L^2 int_0^L int_0^L g(x - x') exp(2 pi i (D1 x + D2 x') / L)
 * dx dx', g(u) = sqrt(pi / alpha) exp(-u^2 / (4 alpha)), for the pair differences
 * D1 = J_x - I_x at r and D2 = L_x - K_x at r').  A is real, symmetric in (D1, D2) and even
 * under (D1, D2) -> (-D1, -D2), so only the canonical pairs d1 >= |d2| are stored, at code
 * c = d1^2 + d1 + d2 (0 <= d1 <= 2R); any (D1, D2) maps to (d1, d2) by swapping so that
 * |D1| >= |D2| and then negating both if the first is negative.  D1 + D2 = 0 entries equal
 * the conserving table of cc_tables_values.  Built with the same 1200-point Gauss-Legendre
 * rule per axis integral as the conserving table.  CC_ERR_NOTSUPP for PERIODIC tables. */
cc_status cc_tables_general_values(cc_tables t, double* table_host);

/* Checkpoint: write / read the node set and the FP64 tables (the "stored forever"
 * table of Sec. II) to a flat versioned file with a checksum.  Load rebuilds the
 * derived device tables on the current device.  CC_ERR_IO on a bad file. */
cc_status cc_tables_save(cc_tables t, const char* path);
cc_status cc_tables_load(const char* path, void* stream, cc_tables* out);

cc_status cc_tables_free(cc_tables t);

/* The mesh (n_sub, q_tail) that cc_build_tables picks when both are left negative, for
 * S nodes at cutoff R (host only, no GPU): see the default rule above. */
cc_status cc_default_mesh(int S, int R, int* n_sub, int* q_tail);

/* Fewest nodes for a stated method error (host only, no GPU; Sec. II: the node count
 * follows from the accuracy wanted over the range of |q|^2 the cutoff R allows).  Returns
 * in *S the smallest S in 2 .. S_max whose default mesh (n_sub, q_tail), as chosen by the
 * default rule above, has a periodic-kernel error max_m |sum_s w_s exp(-a_s m) - 1/m| m
 * (the 96 points of the default rule) of at most target, with that mesh in *n_sub,
 * *q_tail and its error in *err (if not NULL).  Errors below about 1e-10 are FP64
 * rounding noise.  CC_ERR_ARG for NULL outputs or a target that is not positive and
 * finite; CC_ERR_RANGE for R outside 1 .. 127, S_max outside 2 .. 1024, or when no S up to
 * S_max reaches the target. */
cc_status cc_mesh_for_error(int R, double target, int S_max, int* S, int* n_sub, int* q_tail,
                            double* err);

/* Mesh tuning for a stated method error (host only, no GPU; not a rule of the paper, which
 * fixes alpha_c = 1 and leaves "the value of alpha_c which allows for the most efficient
 * numerical integration" and more than two intervals open, Sec. II).  Searches the
 * sub-interval ratio in {3, 4, 5, 6, 8}, alpha_c in {0.5, 1, 2} (periodic index units) and
 * the default rule's n_sub (computed from the ratio) and q_tail ranges, for node counts from
 * 0.8 to 1 times the count cc_mesh_for_error returns for the same target: the fewest nodes
 * whose best candidate has the periodic-kernel error (as in cc_mesh_for_error) of at most
 * target; ties as in the default rule.  Writes the mesh (S, n_sub, q_tail, alpha_c, ratio)
 * and, if err is not NULL, its error.  Errors as cc_mesh_for_error. */
cc_status cc_mesh_tune(int R, double target, int S_max, int* S, int* n_sub, int* q_tail,
                       double* alpha_c, double* ratio, double* err);

/* Build tables (as cc_build_tables, default pruning) on the mesh cc_mesh_tune picks for a
 * stated periodic-kernel method error: the fewest nodes, so the separable lookups and the
 * mode products do the least work for that accuracy.  The box kernel uses the same mesh.
 * Errors as cc_mesh_tune and cc_build_tables. */
cc_status cc_build_tables_for_error(int kernel, int R, double L, double target, int S_max,
                                    void* stream, cc_tables* out);

/* Basis of cutoff R (Sec. II Eq. 1 with |n|^2 <= R^2) in canonical order.  Writes the
 * count to *Nb; if vec_host is not NULL it must hold 4 * Nb int8 and receives
 * (n_x, n_y, n_z, 0) per function.  1 <= R <= 127. */
cc_status cc_basis(int R, int* Nb, int8_t* vec_host);

/* Reconstruct (IJ|KL) for n quadruples (Sec. II Eq. 14; momentum conservation Sec. III).
 *   quads_dev     n quadruples in `format` (16 bytes each and 16-byte aligned; 8 bytes and
 *                 8-byte aligned for CC_QUAD_IDS_U16, which needs Nb <= 65536, else
 *                 CC_ERR_RANGE).
 *   lookup        CC_LOOKUP_SEPARABLE (any kernel), CC_LOOKUP_COLLAPSED (PERIODIC) or
 *                 CC_LOOKUP_GENERAL (BOX): see below.
 *   precision     CC_PREC_FP32 (out float[n]) or CC_PREC_FP64 (out double[n]).
 *   counters_dev  NULL or unsigned long long[3], ADDED to (not cleared):
 *                 [0] non-conserving quadruples, [1] periodic q = 0 (excluded) terms,
 *                 [2] ids outside [0, Nb) or vectors outside the cutoff sphere.
 *                 Each of these quadruples gets the value 0.
 *   BOX kernel, SEPARABLE: the one-index per-axis tables represent momentum-conserving
 *   quadruples only; non-conserving ones get 0 and are counted in [0].
 *   BOX kernel, GENERAL: every in-range quadruple gets its value, conserving or not,
 *   (IJ|KL) = 1/(2 pi^2) sum_s w_s prod_{x,y,z} A(alpha_s, D1, D2) with D1 = n_J - n_I and
 *   D2 = n_L - n_K per axis (Sec. II Eqs. 8 and 14; the two-index tables of
 *   cc_tables_general_values, FP32 or FP64 by precision); [0] still counts the
 *   non-conserving ones (informational, their values are not zeroed), [1] stays 0.
 *   The box integrand changes sign, so a node sum can cancel: an FP32 result is accurate
 *   to about 1e-7 of sum_s |w_s prod A| (the sum of the absolute terms), not of itself.
 * n may be 0.  Errors: CC_ERR_ARG, CC_ERR_NOTSUPP (collapsed BOX, general PERIODIC,
 * mixed precision). */
cc_status cc_reconstruct_integrals(cc_tables t, const void* quads_dev, int64_t n, int format,
                                   int lookup, int precision, void* out_dev,
                                   unsigned long long* counters_dev, void* stream);

/* How the lookups find the index vectors of ids (uint16 or int32) when the basis cannot be
 * staged in shared memory with their table (collapsed: basis and table over 48 KB, R >= 15
 * in FP32, R >= 14 in FP64; separable: over 96 KB; not part of the paper, a comparison
 * switch of this implementation, process-wide): 1 (the default) = decoded on chip from a
 * table of one 32-bit hint per 32 ids staged in shared memory (the line (n_x, n_y) and
 * place of the bucket's first id in the lexicographic basis order of Sec. III, and the next
 * line's length; ids further on walk over whole lines), when table and hints fit in 200 KB
 * (collapsed FP32 up to R = 63, FP64 up to R = 57; separable FP32 at R = 63 with up to 128
 * padded nodes); 0 = a gather from the basis table in global memory.  Results are
 * identical.  CC_ERR_ARG for any other value. */
cc_status cc_set_id_decode(int on);

/* Exchange-type pair integrals (ij|ji) = V(n_j - n_i) for basis rows
 * i = row0 .. row0 + nrows - 1 and every column j:  out_dev[nrows][Nb] (float or double
 * by precision), row major.  Diagonal of the PERIODIC kernel: 0 (q = 0 excluded). */
cc_status cc_pair_matrix(cc_tables t, int64_t row0, int64_t nrows, int lookup, int precision,
                         void* out_dev, void* stream);

/* Exchange sums of the uniform electron gas (Sec. III):
 *   eps(k) = -sum_{j in F} V(k - n_j) on the (2R+1)^3 grid k in [-R, R]^3, row major
 *   [k_x + R][k_y + R][k_z + R], 0 outside the basis sphere |k| <= R.  F is the Fermi
 *   sphere |n| <= R_F (1 <= R_F <= R).  PERIODIC excludes j = k, BOX includes it.
 *   Computed as mode products of the occupation tensor with the Toeplitz matrices
 *   T_s[a][b] = T_s[|a - b|] along x, y and z, accumulated over the nodes s.
 *   Ex_dev[0] = E_x^sigma = 1/2 sum_{k in F} eps(k) (per spin, FP64 reduction),
 *   Ex_dev[1] = 2 E_x^sigma (unpolarised total).
 *   precision: CC_PREC_FP64 / CC_PREC_FP32 (eps double / float, SIMT), CC_PREC_BF16X3 /
 *   CC_PREC_FP16X3 (eps float, tcgen05 tensor cores).  Uses the handle's workspace:
 *   calls on one handle must not overlap on the GPU. */
cc_status cc_exchange_sums(cc_tables t, int R_F, int precision, void* eps_dev, double* Ex_dev,
                           void* stream);

/* Exchange sums without any allocation (no counterpart in the paper).  For callers that
 * cannot call cudaMalloc at the point where they need the sums: code running under a
 * framework's caching allocator that owns the device memory, or latency-critical loops
 * where cudaMalloc's implicit device synchronisation would stall other streams.
 * Computes the same sums as cc_exchange_sums with CC_PREC_FP32 (eps float[Mg^3], Ex_dev[2]),
 * within that call's FP32 tolerance, by the plain chain of SIMT mode products over the
 * handle's tables (cc_exchange_sums may take another FP32 form with another summation
 * order, so the two agree to rounding, not bit for bit), but keeps all scratch in one fixed
 * 16 MiB device array inside the library (held by every GPU that loads the library until
 * the process exits) and calls no cudaMalloc, cudaFree or allocating library routine.
 * Limit: R <= 31 (grid side 63); larger handles get CC_ERR_RANGE.  The handle's device
 * must be the current device (CC_ERR_ARG otherwise).
 * Building or loading a handle of R <= 31 looks up the device's address of the array
 * (cudaGetSymbolAddress, device current), which under CUDA's lazy module loading is what
 * allocates it, and loads the chain's kernels, so that the calls themselves do neither;
 * the address is cached for the rest of the process (the cache assumes the device's
 * primary context lives as long as the process: after a cudaDeviceReset it is stale).
 * Every call shares the array and leaves the last call's contents in it:
 * calls that overlap on the GPU (any device-side overlap, on any stream, from any
 * thread) race and must be ordered by the caller. */
cc_status cc_exchange_sums_noalloc(cc_tables t, int R_F, float* eps_dev, double* Ex_dev,
                                   void* stream);

/* Error word of the tensor-core (mixed precision) exchange path: 0 = fine; 1, 2, 3, 4 = a
 * bounded wait inside the kernel ran out (TMA producer, MMA issuer on its operands,
 * epilogue, MMA issuer on a free accumulator), 5 = the stall of cc_test_stall_next_mixed;
 * the kernel returned without finishing (outputs invalid).  Synchronises; clear != 0 resets
 * it.  Returns CC_ERR_TIMEOUT when the word is nonzero. */
cc_status cc_mixed_status(cc_tables t, int* code_host, int clear);

/* Test hook for the bounded waits (no counterpart in the paper): the next tensor-core
 * GEMM launch of this process makes its MMA warp wait on a barrier that nothing arrives
 * at; after 20 ms the wait gives up, the kernel writes error code 5 to the mixed-path
 * error word (see cc_mixed_status), every role of the CTA stops, TMEM is freed and the
 * kernel returns.  The results of that exchange call are invalid; the context and
 * later calls are not affected. */
cc_status cc_test_stall_next_mixed(void);

/* Which form the tensor-core exchange (bf16x3, fp16x3) takes (not part of the paper; a
 * diagnostic and tuning switch of this implementation, process-wide): 0 = automatic, 1 = the
 * step chain of five batched GEMM launches, 2 = the 128-row fused slab kernel (every grid
 * side up to 127), 3 = the small-grid kernel (bf16x3, grid sides up to 64, two slabs per
 * 128-row MMA; CC_ERR_NOTSUPP for larger grids).  Automatic takes the small-grid kernel for
 * bf16x3 grids up to 64 and the 128-row kernel otherwise (fp16x3: always the 128-row
 * kernel); batches (bf16x3, grid sides up to 49) take the batched small-grid kernel, or
 * the chain on 1.  The setting is read when a batch's graph is captured.  CC_ERR_ARG for any
 * other value. */
cc_status cc_set_mixed_variant(int variant);

/* Split products per mode product in the single-box bf16x3 tensor-core exchange (through
 * the slab kernels; not part of the paper, a diagnostic of this implementation,
 * process-wide): 3 (the default) = hi*hi + hi*lo + lo*hi, where the lo planes carry the
 * rounding residual of every 16-bit operand and correct the product; 1 = hi*hi only, the
 * uncorrected bf16 product, to state what the correction buys (its error is a few 1e-4
 * relative).  fp16x3, batches and the step chain always use 3.  CC_ERR_ARG otherwise. */
cc_status cc_set_mixed_terms(int terms);

/* Which form the plain FP32 exchange (cc_exchange_sums with CC_PREC_FP32) takes at grid
 * sides 50..127 (not part of the paper; a diagnostic and comparison switch of this
 * implementation, process-wide): 0 = automatic, the slab algorithm on the SIMT cores (the
 * first mode product as window sums of the Fermi sphere's lines, the other two restricted
 * to the band |y - R|, |z - R| <= R_F where they do not vanish; the same algorithm as the
 * tensor-core slab kernel, in FP32 with Kahan-compensated node sums); 1 = the dense chain
 * of strided batched SIMT GEMMs over the full grid (eight Mg^4 flop per node).  Smaller
 * grids always take the fused per-node kernel.  CC_ERR_ARG for any other value. */
cc_status cc_set_simt_variant(int variant);

/* Tile shapes of the SIMT mode products of the dense GEMM chain (plain FP32 / FP64 exchange
 * path where it takes the chain): small_tile for the Mg x Mg batched products, large_tile
 * for the products with an Mg^2-long side, each 0 = 64x64, 1 = 32x32, 2 = 64x32 outputs per
 * CTA; threshold = grid side up to which 32x32 tiles are used (< 0 keeps it).  Process-wide
 * default; a choice measured by cc_autotune_gemm for a grid side takes precedence.  Not part
 * of the paper (a tuning knob of this implementation). */
cc_status cc_set_gemm_tiles(int precision, int small_tile, int large_tile, int threshold);

/* Autotuner of those tiles (not part of the paper): runs the dense chain of the handle's mode
 * products (FP32 or FP64, Fermi radius R_F) with each of the 9 (small, large) tile pairs,
 * `reps` timed calls each (CUDA events on `stream`, median), and keeps the fastest pair for
 * this grid side and precision, process-wide.  choice_host[2] (or NULL) receives it, *ms_host
 * (or NULL) its time.  Synchronous; allocates a scratch output.  CC_ERR_ARG / CC_ERR_RANGE
 * for bad arguments. */
cc_status cc_autotune_gemm(cc_tables t, int precision, int R_F, int reps, int* choice_host,
                           float* ms_host, void* stream);

/* The tile pair cc_autotune_gemm measured for a grid side Mg (0 <= Mg < 256) and precision,
 * or -1, -1 when none has been measured in this process. */
cc_status cc_gemm_tiles_tuned(int precision, int Mg, int* small_tile, int* large_tile);

/* ---- batched engine: many independent boxes in one persistent, graph-captured launch.
 * Box i has its own cutoff, side, node count and mesh (p, any kernel; defaults as in
 * cc_build_tables) and Fermi radius R_F (1 <= R_F <= p.R); grid side 2 p.R + 1 <= 49.
 * Exchange sums of every box (Sec. III) come from one launch that takes work items
 * (box, x slab, group of nodes) from an atomic counter, longest first; the last CTA to
 * finish a slab writes that slab of eps, the last to finish a box its E_x.  The first call for a given (precision, eps_dev,
 * Ex_dev) captures the launch in a CUDA graph, later calls replay it. */
typedef struct {
  cc_table_params p;
  int R_F;
} cc_box;
typedef struct cc_batch_s* cc_batch;

/* Build the tables of every box and the launch plan.  Synchronous; owns device memory. */
cc_status cc_batch_create(const cc_box* boxes_host, int nbox, void* stream, cc_batch* out);

/* nbox; eps_offsets_host[nbox + 1] (element offset of box i's (2R_i+1)^3 block in eps_dev,
 * last entry = total); number of work items; device bytes.  Any pointer may be NULL. */
cc_status cc_batch_info(cc_batch b, int* nbox, long long* eps_offsets_host, int* n_items,
                        size_t* device_bytes);

/* Exchange sums of all boxes: eps_dev (double for CC_PREC_FP64, float for CC_PREC_FP32
 * and CC_PREC_BF16X3) holds every box's grid at its offset, Ex_dev[2 i], Ex_dev[2 i + 1] =
 * E_x^sigma and total of box i.  Stream ordered; calls on one batch must not overlap.
 * CC_PREC_BF16X3 (periodic boxes only) runs every box through one launch of the
 * small-grid tensor-core kernel (two slabs per 128-row MMA; work units (box, slab pair,
 * node) cut among one CTA per SM) and one finalising launch, both in the captured graph
 * (cc_set_mixed_variant selects the 128-row slab kernel or the step chain instead); its
 * first call builds the bf16 planes and buffers (synchronous, allocates), later calls
 * allocate nothing. */
cc_status cc_batch_exchange(cc_batch b, int precision, void* eps_dev, double* Ex_dev,
                            void* stream);

/* Launch shape: CTAs per SM (1..16) and oversubscription (1..64): the plan cuts the
 * boxes into about (#SMs x CTAs per SM x oversubscription) work items (x slab x node
 * group), in proportion to each box's cost.  Drops captured graphs. */
cc_status cc_batch_set_plan(cc_batch b, int ctas_per_sm, int oversub);

/* Autotuner.  CC_PREC_FP32 / CC_PREC_FP64 (the SIMT engine): times every launch shape (CTAs
 * per SM in {2, 4, 8}, oversubscription in {1, 2, 4}) and keeps the fastest; choice_host[2]
 * = (CTAs per SM, oversubscription).  CC_PREC_BF16X3 (the tensor-core engine): times every
 * work decomposition, box order (0 as given, 1 by decreasing cost) x cut of the unit
 * sequence among the CTAs (0 equal unit counts, 1 equal estimated cost), and keeps the
 * fastest; choice_host[2] = (order, cut).  CUDA events, median of `reps` runs each;
 * *ms_host receives the best time.  Writes eps_dev / Ex_dev (valid sums) while timing and
 * drops the batch's captured graphs.  Synchronous. */
cc_status cc_batch_tune(cc_batch b, int precision, void* eps_dev, double* Ex_dev, int reps,
                        int* choice_host, float* ms_host, void* stream);

cc_status cc_batch_free(cc_batch b);

/* Human-readable name of a status; detail of the last CUDA failure of this thread. */
const char* cc_status_string(cc_status s);
const char* cc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* COULOMB_H_ */

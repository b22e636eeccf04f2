/*
 * qxd.h -- C ABI of libqxd: the O(a)-improved QCD+QED Wilson-clover Dirac operator on one
 * GB300 (sm_103a), its even-odd Schur complement, and solvers for D psi = eta.
 *
 * Operator (the method's operator, Sec. 1-2 and Sec. 4.3 of arXiv:2502.02490):
 *   D = (4 + m0) - 1/2 sum_mu [ (1 - gamma_mu) W_mu(x) delta_{x+mu,y}
 *                              + (1 + gamma_mu) W_mu(x-mu)^dag delta_{x-mu,y} ]
 *       + c_sw (i/4) sigma_{mu nu} Fhat^SU(3)_{mu nu} + q c_sw^QED (i/4) sigma_{mu nu} Fhat^U(1)_{mu nu}
 *   with U(3) hop links W_mu(x) = exp(i q A_mu(x)) U_mu(x)  (Sec. 4.3).
 *
 * Conventions (all fixed; they are the readings the CPU oracle also uses):
 *   - chiral gamma basis, gamma5 = diag(1,1,-1,-1); clover block 0 (+) acts on spins 0,1;
 *   - Fhat = (Q_{mu nu} - Q_{nu mu}) / 8 from the four plaquette leaves; SU(3) part traceless,
 *     U(1) part from the unit-charge phases exp(iA), multiplied by q;
 *   - 4 + m0 sits in the clover blocks A(x); antiperiodic time = -1 on hops across t=T-1 <-> 0;
 *   - Schur complement Dhat = A_ee - 1/4 H_eo A_oo^-1 H_oe (= D_ee - D_eo D_oo^-1 D_oe).
 *
 * Site orders at the boundary (Sec. 4.1.1):
 *   QXD_ORDER_LEXI : lexicographic Lambda(x, L) = L3 L2 L1 x0 + L3 L2 x1 + L3 x2 + x3 (Eq. lexi),
 *                    i.e. C-contiguous over (t, x, y, z).
 *   QXD_ORDER_IPT  : openQxD order (Eq. ipt): even sites first; within a parity the cache blocks
 *                    of extents B (qxd_set_ipt_blocks; default B = L, one block) in
 *                    lexicographic block order, the sites of a block lexicographic within it.
 *                    With B = L each parity is in floor(Lambda/2) order.
 *   "Even half" vectors (apply_Dhat_eo, solver internals) always list the V/2 even sites in
 *   floor(Lambda/2) order, which is the first half of QXD_ORDER_IPT with one cache block.
 *
 * Field layouts (all doubles, complex numbers interleaved re, im; site order as above):
 *   spinor  [V][4 spin][3 colour][2]          (x, alpha, a) with a fastest (Sec. 2)
 *   links   [V][4 mu][3 row][3 col][2]        forward links mu = 0..3 = t,x,y,z, row-major (Sec. 4.1.4)
 *   angles  [V][4 mu]                         U(1) field A_mu(x)
 *   clover  [V][2 chirality][36]              6 real diagonal entries, then (re, im) of the 15
 *                                             strictly-upper entries in row-major order (Sec. 4.1.3);
 *                                             within a block the index is 3*alpha' + a, alpha' in {0,1}
 *
 * C* boundaries (Sec. 4.2): a lattice created with cstar = 1 is doubled in x, so all spinors
 * live on (T, 2 L1, L2, L3).  load_gauge takes the PHYSICAL field on (T, L1, L2, L3) and builds
 * the charge-conjugated mirror (U -> U*, A -> -A) on the device; a hop across the y or z
 * boundary lands on the mirror copy (x -> x + L1 mod 2 L1).
 *
 * Ownership: the caller owns every pointer it passes.  The library copies what it needs
 * (gauge field at load_gauge) and owns its derived device fields until destroy.
 * on_device = 1: pointers are CUDA device pointers, used on the lattice's stream, and the call
 * returns without a host synchronisation.  on_device = 0: pointers are host memory; the call
 * stages through device buffers and returns after the results are in host memory.
 *
 * Errors: every entry point returns a qxd_status and never exits or aborts.  The message of
 * the last failure on a lattice is in qxd_last_error(lat).
 */
#ifndef QXD_H
#define QXD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qxd_lattice qxd_lattice; /* opaque; owns all device fields of one lattice */
typedef struct qxd_net qxd_net;         /* opaque; a learned preconditioner bound to one lattice */

typedef enum {
  QXD_OK = 0,
  QXD_EINVAL = 1,     /* bad argument: odd or non-positive extent, null pointer, nrhs <= 0, ... */
  QXD_ENOMEM = 2,     /* device allocation failed */
  QXD_ECUDA = 3,      /* a CUDA call failed (message in qxd_last_error) */
  QXD_ESINGULAR = 4,  /* a 6x6 clover block is not invertible (pivot < 1e-14 * max |entry|) */
  QXD_ENOCONV = 5,    /* tolerance not met within maxiter; x holds the best iterate */
  QXD_ESTATE = 6,     /* call out of order, e.g. apply before build_clover */
  QXD_ETIMEOUT = 7    /* a bounded device-side wait expired */
} qxd_status;

typedef enum { QXD_BC_PERIODIC = 0, QXD_BC_ANTIPERIODIC = 1 } qxd_tbc;
typedef enum { QXD_ORDER_LEXI = 0, QXD_ORDER_IPT = 1 } qxd_order;

/* Arithmetic/storage precision of an operator application.
 *   F64  : FP64 fields, FP64 arithmetic.
 *   F32  : FP32 fields, FP32 arithmetic.
 *   F16N : FP16 spinors and clover with one FP32 scale per site (per clover block), FP16 links;
 *          FP32 arithmetic.
 *   BF16N: as F16N with BF16 storage. */
typedef enum { QXD_F64 = 0, QXD_F32 = 1, QXD_F16N = 2, QXD_BF16N = 3 } qxd_prec;

typedef enum {
  QXD_SOLVER_CG_EO = 0,    /* plain FP64 even-odd CG (CG on Dhat^+ Dhat), true-residual judged */
  QXD_SOLVER_MP_CG_EO = 1, /* FP64 outer defect correction around an inner even-odd CG in
                              inner_prec with FP32 reliable updates */
  QXD_SOLVER_MP_BICGSTAB_EO = 2, /* as MP_CG_EO with BiCGStab on Dhat as the inner solver (each
                                   reliable update restarts it from the recomputed residual) */
  QXD_SOLVER_MP_FGCR_NET = 3,    /* FP64 outer defect correction around flexible GCR(gcr_restart) on
                                   the full D in FP32 with the learned network `net` as right
                                   preconditioner (net NULL: no preconditioner) */
  QXD_SOLVER_MP_SAP_GCR = 4,     /* as MP_FGCR_NET with the Schwarz alternating procedure as the
                                   preconditioner (sap_block, sap_ncy, sap_nmr; qxd_sap_apply) */
  QXD_SOLVER_MP_CGNR = 5,        /* FP64 outer defect correction around CG on the normal equations
                                   (D M)^+ D M y = (D M)^+ r of the full lattice in FP32, x += M y,
                                   with the learned network `net` as M (NULL: M = 1) and its adjoint
                                   network as M^+; FP32 reliable updates (reliable_delta).  Converges
                                   for any invertible D, also where D is indefinite and GCR or
                                   BiCGStab stagnate or break down; inner_prec is not used */
  QXD_SOLVER_MP_DFL_SAP_GCR = 6, /* as MP_SAP_GCR with the two-level preconditioner of inexact
                                   deflation: z = P A^-1 P^+ r on the subspace of qxd_dfl_setup
                                   (coarse GCR to its coarse_tol), then z += M_SAP (r - D z)
                                   (QXD_ESTATE without a subspace set up on the current field) */
  QXD_SOLVER_MP_MG_GCR = 7       /* as MP_SAP_GCR with the three-level multigrid preconditioner of
                                   qxd_mg_setup (the deflation subspace as level 1, its aggregation
                                   as level 2; SAP smoothing on the fine lattice with sap_block,
                                   sap_ncy cycles after and the set-up's ncy_pre cycles before the
                                   coarse correction, sap_nmr MR steps per block solve); QXD_ESTATE
                                   without a multigrid set up on the current deflation subspace */
} qxd_solver;

typedef struct {
  int version;            /* must be QXD_PARAMS_VERSION */
  int solver;             /* qxd_solver */
  double tol;             /* target true relative residual ||eta - D psi|| / ||eta|| (e.g. 1e-10) */
  int maxiter;            /* cap on inner iterations summed over all outer rounds */
  int inner_prec;         /* qxd_prec of the inner iteration (MP_CG_EO) */
  double inner_tol;       /* relative reduction asked of each inner solve (MP_CG_EO), e.g. 1e-5 */
  double reliable_delta;  /* reliable update when ||s|| < delta * max||s|| since the last one */
  int max_outer;          /* cap on outer (defect-correction) rounds */
  int on_device;          /* x and b are device (1) or host (0) pointers */
  int check_every;        /* read the residual norm back every this many iterations (>= 1) */
  int gcr_restart;        /* FGCR restart length (MP_FGCR_NET), 1..32 */
  const qxd_net *net;     /* preconditioner of MP_FGCR_NET, or NULL */
  int gcr_reorth;         /* MP_FGCR_NET: classical Gram-Schmidt passes per step, 1 or 2 */
  int fallback;           /* solver run when the solve misses the tolerance (QXD_SOLVER_CG_EO,
                             MP_CG_EO or MP_BICGSTAB_EO, with the library defaults except tol,
                             on_device, check_every; it continues from the failed solve's x when
                             that x has a finite residual below ||b||), or -1 for none */
  /* version 4 */
  int use_x0;             /* 1: x holds an initial guess on entry (same layout as b) and the
                             defect correction starts from r = b - D x (resume from a stored
                             solution); 0: start from x = 0.  qxd_solve only. */
  int restart_f32;        /* 1: when an MP solve with a 16-bit inner_prec misses the tolerance
                             (stagnation, breakdown), restart it once from its current x with
                             FP32 inner precision, a fresh max_outer and the iterations left of
                             maxiter; before any fallback.  qxd_solve only. */
  /* version 5 */
  int sap_block[4];       /* MP_SAP_GCR: block extents (see qxd_sap_apply) */
  int sap_ncy;            /* MP_SAP_GCR: SAP cycles per preconditioner application (>= 1) */
  int sap_nmr;            /* MP_SAP_GCR: minimal-residual steps per block solve (>= 1) */
} qxd_solve_params;

/* Version 4 appended use_x0 and restart_f32, version 5 the SAP fields.  Older structs (version
 * 3 ends at fallback, version 4 at restart_f32) are still accepted: the fields they lack take
 * the defaults, except use_x0 and restart_f32, which a version-3 struct runs with off. */
#define QXD_PARAMS_VERSION 5

typedef struct {
  int iters_inner;        /* inner iterations summed over outer rounds */
  int iters_outer;        /* outer rounds (defect corrections) */
  int reliable_updates;   /* reliable updates performed */
  double true_rel_res;    /* final ||eta - D psi|| / ||eta|| computed in FP64 on the GPU */
  double seconds;         /* wall time of the solve */
  int status;             /* qxd_status of the solve */
  int fallback_used;      /* bit 0 (1): the fallback solver produced x (counts above are then its
                             own); bit 1 (2): the FP32-inner restart ran (counts above include it) */
} qxd_solve_info;

/* Create a lattice of extents L = {T, L1, L2, L3} (txyz, Sec. 4.1.1), all even and >= 2.
 * tbc: time boundary (qxd_tbc).  cstar: 0, or 1 for C* in x, y, z by x-doubling (Sec. 4.2).
 * order: qxd_order of every site-indexed array passed to this lattice.
 * cuda_stream: the cudaStream_t all work is enqueued on (NULL = legacy default stream).
 * On success *out owns its device memory until qxd_destroy_lattice. */
qxd_status qxd_create_lattice(const int L[4], int tbc, int cstar, int order, void *cuda_stream,
                              qxd_lattice **out);

/* Free every device buffer of the lattice; NULL is a no-op. */
qxd_status qxd_destroy_lattice(qxd_lattice *lat);

/* Load the gauge field (Sec. 4.1.4, Sec. 4.3).  su3: links [Vp][4][3][3][2], a_u1: angles
 * [Vp][4] or NULL (= no U(1) field), q: the quark charge multiplying A in the hop links.
 * Vp is the physical volume (V, or V/2 for a C* lattice, whose mirror half is built here).
 * The library copies the data; the caller's arrays are not referenced after return.
 * Invalidates a previously built clover field. */
qxd_status qxd_load_gauge(qxd_lattice *lat, const double *su3, const double *a_u1, double q,
                          int on_device);

/* Update n links of the resident gauge field on the device, without reloading it (the Markov
 * chain changes the field in place; Sec. 6 asks for fields kept on the GPU and updated there).
 *   idx[j]: the link's entry 4 s + mu of the canonical arrays qxd_load_gauge takes (s: the
 *           site on the physical lattice, in the lattice's site order), 0 <= idx[j] < 4 V;
 *   su3:    [n][3][3][2] its new SU(3) (or U(3)) matrix; a_u1: [n] its new U(1) angle, or NULL
 *           for 0.  All three are device pointers with on_device = 1, else host memory.
 * Each link's device copies (two with C*: the mirror one conjugated, angle negated) and its hop
 * link W = exp(i q A) U in every precision are replaced.  If the clover term was built, it is
 * rebuilt (with the m0, c_sw and c_sw^QED of the last qxd_build_clover) at the sites whose
 * plaquettes hold an updated link -- the link's two end points and their +-nu neighbours -- or in
 * full when that is most of the lattice.  Entries of idx must be distinct (with a repeated link
 * it is unspecified which value wins).  Synchronises the lattice stream.  Errors: QXD_ESTATE
 * before load_gauge; QXD_EINVAL for n < 0, a null pointer or an index outside the range (the
 * other links are updated; the clover is then marked unbuilt, so applies return QXD_ESTATE until
 * qxd_build_clover); QXD_ESINGULAR if a rebuilt odd-site
 * block is not invertible (the clover must then be rebuilt before the next apply). */
qxd_status qxd_update_links(qxd_lattice *lat, int64_t n, const int64_t *idx, const double *su3,
                            const double *a_u1, int on_device);

/* Cache blocks of QXD_ORDER_IPT (Eq. ipt, Sec. 4.1.1): B[mu] must divide the lattice extent L[mu]
 * (for C* both the physical and the doubled x extent); default B = L.  Applies to every field
 * exchanged afterwards (spinors, gauge field, clover export).  QXD_EINVAL for a LEXI lattice or
 * a B that does not tile the lattice. */
qxd_status qxd_set_ipt_blocks(qxd_lattice *lat, const int B[4]);

/* Load the gauge field in openQxD's storage (Sec. 4.1.4): for each odd site x, in the order of
 * its index x^ in Eq. ipt (odd sites are x^ = V/2 .. V-1), eight links: u8[8 (x^ - V/2) + 2 mu] =
 * U_mu(x) and u8[8 (x^ - V/2) + 2 mu + 1] = U_mu(x - mu), each 3x3 row-major complex; every link
 * of the lattice appears exactly once (each has one odd end).  u8: [V/2][8][3][3][2]; a8 (or
 * NULL): the U(1) angles in the same arrangement, [V/2][8].  The field is the lattice's own: for
 * C* the doubled lattice with its mirror half (no mirroring is done).  Needs QXD_ORDER_IPT.
 * Otherwise as qxd_load_gauge. */
qxd_status qxd_load_gauge_openqxd(qxd_lattice *lat, const double *u8, const double *a8, double q,
                                  int on_device);

/* Build the clover blocks A(x) = (4+m0) + c_sw (i/4) sigma.Fhat^SU(3) + q c_sw^QED (i/4)
 * sigma.Fhat^U(1) on every site (Sec. 2, Sec. 4.1.3, Sec. 4.3, Sec. 6: clover generated on the
 * GPU) and their inverses on odd sites (6x6 Gauss-Jordan with partial pivoting, FP64), plus
 * the FP32 / FP16 copies the low-precision operators use.
 * Returns QXD_ESINGULAR if some odd-site block has a pivot below 1e-14 times its largest entry;
 * QXD_ESTATE before load_gauge. */
qxd_status qxd_build_clover(qxd_lattice *lat, double m0, double csw, double csw_qed);

/* Copy the FP64 clover field out as [V][2][36] (packing of Sec. 4.1.3), site order of the
 * lattice.  QXD_ESTATE before build_clover. */
qxd_status qxd_get_clover(qxd_lattice *lat, double *out, int on_device);

/* out = D in for nrhs right-hand sides: in, out are [nrhs][V][4][3][2] in the lattice's site
 * order.  prec selects the operator's precision (inputs are rounded to it, outputs widened
 * back to FP64).  With nrhs > 1 and prec F32 the multi-RHS kernel applies D to up to 12
 * right-hand sides per link and clover load; with F16N or BF16N the 16-bit multi-RHS kernel
 * stages each tile's links and clover once for a group of right-hand sides.  QXD_ESTATE before build_clover; QXD_EINVAL for nrhs <= 0 or a null pointer. */
qxd_status qxd_apply_D(qxd_lattice *lat, double *out, const double *in, int prec, int nrhs,
                       int on_device);

/* out_e = Dhat in_e (dagger = 0) or Dhat^dag in_e = gamma5 Dhat gamma5 in_e (dagger = 1), with
 * Dhat = A_ee - 1/4 H_eo A_oo^-1 H_oe on even-half vectors [V/2][4][3][2]. */
qxd_status qxd_apply_Dhat_eo(qxd_lattice *lat, double *out_e, const double *in_e, int prec,
                             int dagger, int on_device);

/* Solve D x = b to the true relative residual params->tol (x is overwritten; the solve starts
 * from zero, or from x itself with params->use_x0).  b, x: [V][4][3][2].  info (may be NULL)
 * receives iteration counts, the final FP64 true residual and the wall time.  Recovery when the
 * tolerance is missed: the FP32-inner restart (restart_f32), then the fallback solver
 * (fallback).  QXD_ENOCONV when the tolerance is still not met; x then holds the last iterate. */
qxd_status qxd_solve(qxd_lattice *lat, double *x, const double *b, const qxd_solve_params *params,
                     qxd_solve_info *info);

/* Solve D x_r = b_r for nrhs right-hand sides in lock step (e.g. the 12 spin-colour point
 * sources of a propagator): FP64 outer defect correction per right-hand side and one inner
 * BiCGStab (FP32 vectors) over all of them whose Dhat applications load each site's links and
 * clover once for every right-hand side (inner_prec F32: FP32 fields; F16N / BF16N: 16-bit
 * spinors, links and clover with per-site norms, FP32 reliable updates).
 * x, b: [nrhs][V][4][3][2]; info: nrhs entries (or NULL).
 * params: solver MP_BICGSTAB_EO, inner_prec F32, F16N or BF16N, use_x0 0 (else QXD_EINVAL); fallback and
 * restart_f32 are not used; the other fields as for qxd_solve.  QXD_ENOCONV if some right-hand
 * side misses the tolerance. */
qxd_status qxd_solve_mrhs(qxd_lattice *lat, double *x, const double *b, int nrhs,
                          const qxd_solve_params *params, qxd_solve_info *info);

/* Solve D_k x_k = b_k for n <= 16 independent lattices (uneven volumes allowed) in one go: per
 * lattice the FP64 outer defect correction of MP_BICGSTAB_EO, and ONE cooperative persistent
 * kernel running the FP32 inner BiCGStab of all lattices together over a work list of site
 * tiles, with bounded-wait grid barriers (QXD_ETIMEOUT if one expires; nothing hangs).  The
 * inner launch is captured in a CUDA graph and replayed every outer round; the tile shape is
 * autotuned on the first call for a set of volumes and remembered.  lats must share one stream
 * and have their clover built; x[k], b[k] are DEVICE fields [V_k][4][3][2] (params->on_device
 * must be 1); info: n entries (iters_inner per lattice, iters_outer the batch's rounds).  params:
 * tol, maxiter (caps the largest lattice's inner iterations), inner_tol, max_outer as for
 * qxd_solve (solver and inner_prec are implied; use_x0 must be 0; fallback and restart_f32 are
 * not used).  The paper solves one lattice at a time; the
 * batch is a throughput layer over the same even-odd mixed-precision solve (Sec. 3, Sec. 5.1). */
qxd_status qxd_solve_batch(qxd_lattice *const *lats, int n, double *const *x, const double *const *b,
                           const qxd_solve_params *params, qxd_solve_info *info);
/* Tuning cache file of qxd_solve_batch (NULL or "" = none, the default).  A set of volumes not
 * yet tuned in this process is looked up there first; each newly tuned set is appended as the
 * line "qxd-batch-tune 1 <GPU name, spaces as _> <SM count> <V0,V1,...,> <blocks/SM>
 * <sites/thread>".  A missing or unreadable file, and malformed lines, are ignored. */
qxd_status qxd_batch_tune_cache(const char *path);
/* Iteration limit of the persistent kernel's barrier spin-waits (default 2e7, about 1.3 s);
 * a tiny limit makes the waits run out (QXD_ETIMEOUT), for tests of that path. */
qxd_status qxd_batch_set_spin_limit(long long limit);
/* Tile shape and graph use of the last qxd_solve_batch: threads per block, sites per thread,
 * resident blocks per SM of the persistent kernel (1 or 2), graph = 1 if the inner launch ran
 * from a captured CUDA graph. */
qxd_status qxd_batch_last_config(int *threads, int *sites_per_thread, int *blocks_per_sm, int *graph);

/* Fill *p with the defaults: MP_CG_EO, tol 1e-10, maxiter 100000, inner F32, inner_tol 1e-5,
 * reliable_delta 0.1, max_outer 20, on_device 1, check_every 1, gcr_restart 16, net NULL,
 * gcr_reorth 1, fallback -1, use_x0 0, restart_f32 1, sap_block {4, 4, 4, 4}, sap_ncy 2, sap_nmr 4. */
void qxd_default_params(qxd_solve_params *p);

/* out = M in with M the Schwarz alternating procedure (Sec. 5.1 names it as the preconditioner
 * of the paper's CPU solves), on full fields [V][4][3][2], FP32 arithmetic.  The lattice is cut
 * into blocks of extents block[mu] (each divides the lattice extent on the device, x doubled
 * for C*, with an even number of blocks per direction, and for C* the physical L1 an even number
 * of x blocks; at most 256 sites per block), so that blocks of one colour never touch.  A block's
 * colour is the parity of its block coordinates.  Each of ncy cycles sweeps colour 0, then
 * colour 1.  Every block of the colour takes nmr minimal-residual steps from zero on D
 * restricted to the block (hops leaving it dropped) for the current residual; the result is
 * added to the output, and the residual in - D out is recomputed.  QXD_EINVAL for a block shape
 * outside these rules, ncy < 1 or nmr < 1; QXD_ESTATE before build_clover. */
qxd_status qxd_sap_apply(qxd_lattice *lat, double *out, const double *in, const int block[4], int ncy,
                         int nmr, int on_device);

/* Fused BLAS-1 on device vectors of n complex numbers (interleaved re, im), on the lattice's
 * stream, FP64.  Reductions are deterministic (fixed order) and return to host memory.
 * Vectors must be device (or managed) memory aligned to 16 bytes, else QXD_EINVAL.
 * n = 0 is allowed (pointers may then be NULL): dot and norm2 give 0, axpy does nothing.
 *   dot:   *re + i *im = sum_k conj(a_k) b_k
 *   norm2: *out = sum_k |a_k|^2
 *   axpy:  y_k += (re + i im) x_k                                                         */
qxd_status qxd_vec_dot(qxd_lattice *lat, const double *a, const double *b, int64_t n, double *re,
                       double *im);
qxd_status qxd_vec_norm2(qxd_lattice *lat, const double *a, int64_t n, double *out);
qxd_status qxd_vec_axpy(qxd_lattice *lat, double re, double im, const double *x, double *y,
                        int64_t n);

/* ---- Learned preconditioner (gauge-equivariant parallel-transport convolution network) ----
 * Layer: out_c(x) = sum_{c'} sum_{p=0..8} Omega[c][c'][p] (T_p h_{c'})(x) with T_0 = 1,
 * T_{1+mu} h(x) = W_mu(x) h(x+mu), T_{5+mu} h(x) = W_mu(x-mu)^dag h(x-mu) (hop links and
 * boundary conditions of the lattice; gauge-equivariant by construction) and Omega a complex
 * 4x4 spin matrix per (output channel, input channel, path).  The network is the chain of
 * nlayers linear layers with channel counts channels[0..nlayers] (first and last 1, others
 * 1..16).  FP32 weights.  Weights are laid out [layer][Cout][Cin][9][4][4] complex
 * (interleaved re, im doubles at the boundary).  The paper has no learned part; this follows the
 * method's learned-preconditioner extension.
 * create: weights initialised from `seed` (identity path near 1/4, small noise elsewhere). */
qxd_status qxd_net_create(qxd_lattice *lat, int nlayers, const int *channels, uint64_t seed,
                          qxd_net **out);
qxd_status qxd_net_destroy(qxd_net *net);
int64_t qxd_net_num_weights(const qxd_net *net); /* complex weights */
qxd_status qxd_net_set_weights(qxd_net *net, const double *w); /* host [n][2] */
qxd_status qxd_net_get_weights(const qxd_net *net, double *w);
/* out = M^+ in, the adjoint network: the layers last to first, each with the weights
 * Omega[c][c'][p] -> Omega[c][c'][p']^+ of the opposite path p' (the adjoint of the transport along
 * p is the transport along -p, and it commutes with the spin matrices), in the net's precision.
 * <phi, M psi> = <M^+ phi, psi> up to rounding.  Layout and errors as qxd_net_apply. */
qxd_status qxd_net_apply_adjoint(qxd_net *net, double *out, const double *in, int on_device);

/* Inference precision of qxd_net_apply and of the network inside QXD_SOLVER_MP_FGCR_NET:
 * QXD_NET_BF16_TC (default): each layer's channel mix on the tensor cores (tcgen05), BF16
 *   transported activations and weights, FP32 accumulation and FP32 activations between layers;
 * QXD_NET_F32: FP32 on the CUDA cores.  Training (qxd_net_loss_grad, qxd_net_train) always runs
 * in FP32.  QXD_ETIMEOUT from qxd_net_apply if a bounded wait of the tensor-core kernel expired. */
#define QXD_NET_F32 0
#define QXD_NET_BF16_TC 1
qxd_status qxd_net_set_precision(qxd_net *net, int prec);
/* out = M in on full fields [V][4][3][2]. */
qxd_status qxd_net_apply(qxd_net *net, double *out, const double *in, int on_device);
/* loss = sum_i ||M(b_i) - v_i||^2 over nsamp samples ([nsamp][V][4][3][2] each) and, if grad is
 * non-NULL, grad = dloss/d(conj w) (host [n][2]; the real-parameter gradient is twice its real
 * and imaginary parts). */
qxd_status qxd_net_loss_grad(qxd_net *net, const double *v, const double *b, int nsamp, int on_device,
                             double *loss, double *grad);

typedef struct {
  int version;   /* QXD_TRAIN_VERSION (qxd_net_train also takes 1, which ends at eps) */
  int epochs;    /* passes over the training set */
  int batch;     /* samples per Adam step */
  double lr, beta1, beta2, eps; /* Adam */
  /* version 2: read by qxd_train_precond only */
  int nlayers;          /* network depth, as qxd_net_create */
  int channels[9];      /* channels[0..nlayers], as qxd_net_create */
  int nsamp;            /* training pairs generated on the device */
  uint64_t net_seed;    /* weight initialisation, as qxd_net_create */
  uint64_t sample_seed; /* sample i is the Gaussian field of seed sample_seed + i (see below) */
  double *loss_hist;    /* host [epochs]: mean loss per epoch, or NULL */
} qxd_train_params;
#define QXD_TRAIN_VERSION 2

/* Train on (b_i = D v_i, v_i), i < nsamp, generated by the lattice's own FP32 operator from the
 * given v ([nsamp][V][4][3][2], e.g. Gaussian): Adam on sum_i ||M(b_i) - v_i||^2 with the
 * network's own forward and backward kernels.  loss_hist (may be NULL): mean loss per epoch. */
qxd_status qxd_net_train(qxd_net *net, const double *v, int nsamp, const qxd_train_params *p,
                         double *loss_hist, int on_device);
/* Create and train a network in one call, with the training set generated on the device: sample
 * i is the Gaussian spinor v_i whose component (alpha, a) at the site of lexicographic index x
 * (Eq. lexi on the lattice's device extents, x doubled for C*) is re + i im = r (cos th + i sin th)
 * (Box-Muller), r = sqrt(-2 ln(1 - u_{2j})), th = 2 pi u_{2j+1}, j = 12 x + 3 alpha + a, u_n the top
 * 53 bits of SplitMix64 output n of seed sample_seed + i (counter style: mix(seed + (n + 1)
 * 0x9E3779B97F4A7C15)), rounded to FP32; then as qxd_net_train on (D v_i, v_i).  Needs
 * p->version 2; *out owns the network (qxd_net_destroy).  On failure *out is NULL. */
qxd_status qxd_train_precond(qxd_lattice *lat, const qxd_train_params *p, qxd_net **out);
/* Checkpoint: "QXDNET1\n", int32 nlayers, int32 channels[nlayers+1], float32 weights (re, im). */
qxd_status qxd_net_save(const qxd_net *net, const char *path);
qxd_status qxd_net_load(qxd_lattice *lat, const char *path, qxd_net **out);

/* ---- Inexact deflation (the "DFL" of the DFL_SAP_GCR solver of Sec. 5.1; the paper names it
 * without detail, so this is the textbook two-level method) ----
 * qxd_dfl_generate: approximate low modes from ns start fields (the caller draws them): each is
 *   normalised and then improved by n_it normalised SAP inverse iterations v <- M_SAP v / ||.||
 *   (FP32 SAP with blocks sap_block, ncy cycles, nmr MR steps).  start, out: [ns][V][4][3][2].
 * qxd_dfl_setup: the deflation subspace of ns fields `vectors` ([ns][V][4][3][2], host or device
 *   per on_device) on blocks of extents block[4]: restricted to each block and orthonormalised
 *   there (modified Gram-Schmidt in vector order, FP64), and the little Dirac operator
 *   A = P^+ D P (FP64), which couples a block to itself and its eight face neighbours.  Blocks:
 *   each extent divides L, the block grid is 1 or even per direction, extents >= 2 where the grid
 *   has more than one block, at most 256 sites; with C* the physical L1 is an even number of x
 *   blocks and the grid has at least two blocks in y and in z.  The coarse solve of the preconditioner (GCR(16) on A, FP64) stops at
 *   ||f - A c|| <= coarse_tol ||f|| or after coarse_maxiter steps.  Replaces an earlier subspace;
 *   a later load_gauge, build_clover or update_links makes it stale (QXD_ESTATE from the solve).
 *   QXD_EINVAL for a bad block shape, ns outside 1..64 or vectors that are linearly dependent on a
 *   block; QXD_ESTATE before build_clover.
 * qxd_dfl_get_little: A as [nb][9][ns][ns][2] doubles (entry (b, slot, k, k') couples basis vector
 *   k of block b with vector k' of block nbr[b][slot]; slot 0 the block itself, 1 + 2 mu the
 *   neighbour in +mu, 2 + 2 mu in -mu) and nbr [nb][9]; host arrays.  Blocks are numbered
 *   lexicographically by block coordinates (direction 3 fastest).
 * qxd_dfl_info: the number of blocks, ns, and the coarse iterations and coarse solves so far. */
qxd_status qxd_dfl_generate(qxd_lattice *lat, const int sap_block[4], int ncy, int nmr, int ns, int n_it,
                            const double *start, double *out, int on_device);
qxd_status qxd_dfl_setup(qxd_lattice *lat, const int block[4], int ns, const double *vectors, int on_device,
                         double coarse_tol, int coarse_maxiter);
qxd_status qxd_dfl_get_little(qxd_lattice *lat, double *A, int *nbr);
qxd_status qxd_dfl_info(qxd_lattice *lat, int *nblocks, int *ns, int64_t *coarse_iters, int64_t *coarse_calls);

/* Multigrid (Sec. 5.1: the paper's GPU solves use multigrid GCR; the paper gives no detail).
 * Three levels: the fine D; level 1, the little Dirac operator A1 = P1^+ D P1 of the deflation
 * subspace of qxd_dfl_setup (a level-1 vector holds n1 = nblocks * ns complex numbers, entry
 * b * ns + k for block b in the block order of qxd_dfl_get_little and basis vector k); level 2,
 * aggregates of agg[0] x agg[1] x agg[2] x agg[3] level-1 blocks, numbered lexicographically by
 * aggregate coordinates (direction 3 fastest), with a basis of ns2 level-1 vectors orthonormalised
 * on every aggregate (modified Gram-Schmidt in vector order) and A2 = P2^+ A1 P2.  The
 * preconditioner of QXD_SOLVER_MP_MG_GCR, on the FP32 fields of the inner flexible GCR:
 *   z = M_SAP^pre r (ncy_pre cycles; none for 0); z += P1 K1(P1^+ (r - D z)); z += M_SAP (r - D z),
 *   K1  = n1 flexible GCR steps on A1 from zero, each preconditioned by the two-grid cycle
 *   T1 f: y = S1 f; y += P2 G2(P2^+ (f - A1 y)); y += S1 (f - A1 y),
 *   S1  = nu minimal-residual steps on A1 from zero, G2 = n2 GCR steps on A2 from zero.
 * GCR steps (both coarse levels, restart every m): z = M r, w = A z, classical Gram-Schmidt of w
 * against the cycle's earlier normalised w (same combination on z), both divided by ||w||,
 * alpha = <w, r>, x += alpha z, r -= alpha w.  Coarse levels are FP64 with fixed step counts and
 * every coefficient on the device (no host synchronisation inside the preconditioner).
 * qxd_mg_setup: vectors [ns2][n1][2] doubles (host, or device with on_device = 1), copied.
 *   Aggregate extents must divide the deflation block grid, and the aggregates must form a
 *   nearest-neighbour grid (with C*, the x shift across the y and z boundaries a whole number of
 *   aggregates), else QXD_EINVAL; likewise for p->version != QXD_MG_VERSION, a parameter outside
 *   its range or vectors linearly dependent on an aggregate.  QXD_ESTATE without a deflation
 *   subspace on the current field.  Replaces an earlier multigrid; a later qxd_dfl_setup or field
 *   change makes it stale (QXD_ESTATE from the solve and the apply calls).  Synchronises.
 * qxd_mg_generate: level-2 vectors by inverse iteration on level 1: each of the ns2 start vectors
 *   [ns2][n1][2] is normalised, then n_it times replaced by k GCR steps (restart 16) on
 *   A1 v' = v, normalised; the results go to out (same layout).  Needs qxd_dfl_setup only.
 * qxd_mg_get_coarse: A2 as [nb2][9][ns2][ns2][2] doubles (slot 0 the aggregate itself, 1 + 2 mu
 *   the neighbour in +mu, 2 + 2 mu in -mu) and nbr2 [nb2][9]; host arrays.
 * qxd_mg_info: the number of aggregates, ns2 and the level-1 solves K1 run so far.
 * qxd_mg_apply_level1: out = K1(in) for one level-1 vector [n1][2] (FP64 throughout).
 * qxd_mg_precond: out = M_MG in for full fields [V][4][3][2] (boundary site order), the fine part
 *   in FP32 as inside the solver; SAP blocks, ncy (post) and nmr as in qxd_sap_apply. */
#define QXD_MG_VERSION 1
typedef struct {
  int version;    /* QXD_MG_VERSION */
  int agg[4];     /* aggregate extents in deflation blocks */
  int ns2;        /* level-2 vectors (1..32, at most the entries of an aggregate) */
  int nu;         /* MR steps of the level-1 smoother, before and after the coarse correction (0..16) */
  int n1;         /* flexible GCR steps of the level-1 solve K1 (1..64) */
  int n2;         /* GCR steps of the coarsest solve (1..256) */
  int m;          /* restart length of both coarse GCRs (1..16) */
  int ncy_pre;    /* SAP cycles before the coarse correction on the fine lattice (0..8) */
} qxd_mg_params;
qxd_status qxd_mg_setup(qxd_lattice *lat, const qxd_mg_params *p, const double *vectors, int on_device);
qxd_status qxd_mg_generate(qxd_lattice *lat, int ns2, int n_it, int k, const double *start, double *out,
                           int on_device);
qxd_status qxd_mg_get_coarse(qxd_lattice *lat, double *A2, int *nbr2);
qxd_status qxd_mg_info(qxd_lattice *lat, int *nb2, int *ns2, int64_t *level1_solves);
qxd_status qxd_mg_apply_level1(qxd_lattice *lat, double *out, const double *in, int on_device);
qxd_status qxd_mg_precond(qxd_lattice *lat, double *out, const double *in, const int sap_block[4], int ncy,
                          int nmr, int on_device);

/* Dot product for callers that cannot allocate device memory.  The paper has no counterpart:
 * this entry point exists for callers that must not call cudaMalloc -- code inside a framework
 * whose device memory belongs to its own caching allocator, and latency-critical loops that
 * cannot afford the device synchronisation an allocation can cause.
 *   out[0] + i out[1] = sum_k conj(a_k) b_k over n complex numbers (FP64, interleaved re, im).
 * a, b: device vectors; out: DEVICE memory for 2 doubles; cuda_stream: stream to run on (NULL =
 * legacy default stream).  No lattice is needed and the call returns without synchronising.
 * Scratch: a static device array inside the library (64 KiB of per-block partial sums plus a
 * counter), which every GPU that loads the library keeps until process exit.  Limit: n <=
 * QXD_NOALLOC_MAX_N; larger n returns QXD_EINVAL.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the life of the process (make
 * that first call before any stream capture begins); after a cudaDeviceReset on that device the
 * kept address is stale: call qxd_vec_dot_noalloc_forget first, and then make a fresh first call
 * before any capture.  All calls share the one array: calls that overlap on the GPU (e.g. on two
 * streams at once) race and give wrong results; serialise them.  The result is deterministic
 * for a given n (fixed blocking) and agrees with qxd_vec_dot to rounding.  Allocates nothing
 * and calls no allocating routine.  Errors: QXD_EINVAL for n < 0, n > QXD_NOALLOC_MAX_N, a
 * null pointer (a and b may be NULL when n = 0), a pointer that is not device (or managed)
 * memory, a or b not 16-byte aligned, or out not 8-byte aligned; QXD_ECUDA if a CUDA call fails; the message
 * is in qxd_last_error(NULL). */
#define QXD_NOALLOC_MAX_N 16777216
qxd_status qxd_vec_dot_noalloc(const double *a, const double *b, int64_t n, double *out,
                               void *cuda_stream);
/* Drops the scratch addresses qxd_vec_dot_noalloc keeps (all devices), so that its next call
 * looks them up again; for use after a device reset.  Host state only: no CUDA call, no device
 * needed.  Thread-safe (it takes the lock of the lookups); on a device that was not reset it only
 * costs the next call one more lookup.  Always returns QXD_OK. */
qxd_status qxd_vec_dot_noalloc_forget(void);

/* Kernel timing.  With profiling on, the library brackets each launch of its hop kernels with
 * CUDA events on the lattice stream; qxd_kernel_stats returns, for the kernel class `which`
 * (0 = FP64 hop, 1 = FP32 hop, 2 = FP16N hop, 3 = BF16N hop, 4 = FP32 multi-RHS hop, 5 = the
 * persistent batch kernel of qxd_solve_batch, counted on the batch's first lattice, 6 = tensor-core
 * PTC layer, 7 = FP32 PTC layer; bytes of a PTC layer: input channels, links and output channels
 * once per site; 8 = 16-bit multi-RHS hop; 9 = SAP block sweep, bytes: residual, x read and
 * written, links and clover once per site of the colour; 10 = the vector kernels of the multi-RHS
 * BiCGStab, bytes: the FP32 vectors each reads and writes), the number of timed launches, their
 * summed device time in ms and the summed algorithmic bytes they moved.  Reading the stats
 * synchronises the stream.  qxd_launch_count is the number of kernels the library launched. */
qxd_status qxd_set_profiling(qxd_lattice *lat, int on);
qxd_status qxd_kernel_stats(qxd_lattice *lat, int which, int64_t *launches, double *ms,
                            double *bytes);
int64_t qxd_launch_count(const qxd_lattice *lat);

/* Guard words, a memory checker for the tests: every device field and work buffer the lattice
 * allocates carries 256 extra bytes filled with 0xA5 behind its end.  *bad receives the number
 * of those bytes that have changed (0: no kernel wrote past the end of a library buffer); a
 * non-zero count is also recorded in qxd_last_error.  Not guarded: buffers the caller owns, the
 * batch cache of qxd_solve_batch and the buffers of a qxd_net.
 * Synchronises the lattice stream.  QXD_EINVAL for a NULL lattice or bad. */
qxd_status qxd_check_guards(qxd_lattice *lat, int64_t *bad);

/* Message of the last failure on this lattice ("" if none); never NULL.  With lat == NULL,
 * the message of the last failed call made without a lattice (qxd_create_lattice,
 * qxd_vec_dot_noalloc). */
const char *qxd_last_error(const qxd_lattice *lat);

#ifdef __cplusplus
}
#endif

#endif /* QXD_H */

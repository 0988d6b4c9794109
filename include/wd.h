/*
 * wd.h -- C ABI of the Wilson-Dirac operator library (libwd.so) for GB300 (sm_103a).
 *
 * The library applies the Wilson-Dirac operator of arXiv:1810.04201, section 2.1,
 * Eq. (1), and solves D psi = eta (section 2.2, Eq. (4)) by Conjugate Gradient on
 * the normal equations D^dag D x = D^dag b, with the whole solve on the device.
 *
 * Operator (hopping term written with -kappa; the paper prints +kappa, which is
 * the same operator conjugated by eps(n) = (-1)^(x+y+z+t) on even lattices, so
 * the paper's form is obtained by passing -kappa):
 *
 *   (D psi)(n) = psi(n) - kappa sum_mu [ b+_mu(n) (1 - gamma_mu) U_mu(n) psi(n+mu)
 *                                      + b-_mu(n) (1 + gamma_mu) U_mu(n-mu)^dag psi(n-mu) ]
 *
 * gamma_mu are the matrices of the paper's Appendix A (the DeGrand-Rossi chiral
 * basis); mu = 0, 1, 2, 3 = x, y, z, t.  With antiperiodic_t set, b+_3(n) = -1 when
 * n_t = T-1 and b-_3(n) = -1 when n_t = 0 (section 2.3: periodic or antiperiodic
 * boundary conditions); all other b are +1 and the stored links are never changed.
 *
 * Canonical layouts (the boundary format, complex = two doubles re, im):
 *   links   U[mu][n][A][B]          4 x V x 3 x 3 complex128, row A, column B;
 *                                    U_mu(n) on the edge n -> n+mu (section 2.1)
 *   spinors psi[r][n][alpha][A]     nrhs x V x 4 x 3 complex128, spin-major,
 *                                    colour-minor (su3_spinor, section 6.1)
 *   site    n = x + Lx*(y + Ly*(z + Lz*t))
 *
 * Device fields.  The operators and solvers work on "fields": device buffers in
 * the library's site-coalesced structure-of-arrays layout, of wd_field_bytes()
 * bytes, written by wd_pack and read back by wd_unpack.  Per right-hand side:
 *   WD_F64: 12 arrays (one per spin-colour component) of Vs complex128 (16 B);
 *   WD_F32: 6 arrays of Vs float4 (two complex64 components each);
 *   WD_F16: 3 arrays of Vs x 16 B (four half2 components each), then Vs floats
 *           holding the per-site scale (the component of largest magnitude);
 *   WD_DF32: 12 arrays of Vs float4 (re.hi, im.hi, re.lo, im.lo);
 * where Vs is V rounded up to a multiple of 64.  Right-hand sides follow each
 * other at a stride of wd_field_bytes(ctx, prec, 1).  Fields must be 256-byte
 * aligned (torch and cudaMalloc allocations are).
 *
 * Ownership and streams.  The caller owns every field and canonical buffer; the
 * context owns its gauge copies, its workspace and its CUDA graphs, and frees
 * them in wd_destroy.  Every call is asynchronous on the context's stream, except
 * the solvers, which wait for the result to fill wd_cg_result, and the calls
 * whose on_device flag is 0 (host buffers), which return once the host buffer
 * may be reused.
 *
 * Errors.  Every call returns a status and never aborts or throws.  Argument
 * checks (null pointers, dimensions < 2, nrhs outside 1..WD_MAX_RHS, unknown
 * precision, no gauge field set) happen before anything is launched; the message
 * of the last failure is available from wd_last_error.
 */
#ifndef WD_H
#define WD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WD_MAX_RHS 16

typedef enum wd_status {
    WD_OK = 0,
    WD_ERR_ARG = 1,           /* invalid argument; nothing was launched */
    WD_ERR_CUDA = 2,          /* a CUDA call failed; see wd_last_error */
    WD_ERR_OOM = 3,           /* device allocation failed */
    WD_ERR_NOT_CONVERGED = 4, /* solver hit max_iter before the tolerance */
    WD_ERR_BREAKDOWN = 5,     /* CG breakdown: p^dag A p <= 0 or a singular block Gram matrix */
    WD_ERR_NONFINITE = 6,     /* a NaN or Inf appeared in a residual or scalar */
    WD_ERR_TIMEOUT = 7,       /* a bounded device-side wait ran out (batched persistent solver) */
    WD_ERR_STATE = 8          /* call out of order (e.g. no gauge field set) */
} wd_status;

/* Storage and arithmetic precision of a field and of the operator applied to it.
 *   WD_F64   IEEE double.
 *   WD_F32   IEEE single.
 *   WD_F16   half-precision storage with a per-site FP32 scale, FP32 accumulation:
 *            the spin projection adds half values in half precision and the SU(3)
 *            products multiply half values into FP32 sums (exact products).
 *   WD_DF32  double-FP32: every real is the unevaluated sum of two floats (48-bit
 *            significand), stored in the same 16 bytes per complex number as
 *            WD_F64 and computed on the FP32 pipes with error-free transformations
 *            (Knuth TwoSum, FMA TwoProduct).  The exponent range is that of FP32.
 *            The operator matches the FP64 definition to about 1e-14 relative. */
typedef enum wd_prec { WD_F64 = 0, WD_F32 = 1, WD_F16 = 2, WD_DF32 = 3 } wd_prec;

typedef struct wd_ctx wd_ctx;

/* Create a context for an Lx x Ly x Lz x Lt lattice (dims[0..3], each >= 2) on the
 * current CUDA device.  stream is a cudaStream_t (NULL = the legacy default stream);
 * all work of this context is queued on it.  antiperiodic_t selects the antiperiodic
 * time boundary (section 2.3). */
wd_status wd_create(wd_ctx **ctx, const int dims[4], int antiperiodic_t, void *stream);
wd_status wd_destroy(wd_ctx *ctx);
wd_status wd_set_stream(wd_ctx *ctx, void *stream);

/* Load the gauge field (section 2.3: the links stay resident across calls).
 * U_canon: canonical links (4*V*9 complex128), host memory (on_device = 0) or device
 * memory (on_device = 1).  recon = 18 stores all nine entries; recon = 12 stores the
 * first two rows and rebuilds the third as conj(row0 x row1) (section 6.1, valid for
 * SU(3) links only); recon = 8 stores U01, U02, U10 and the phases of U00 and U20 and
 * rebuilds the rest from unitarity and det U = 1 (the reconstruction the paper defers
 * in section 6.1; SU(3) links with |U01|^2 + |U02|^2 >= 1e-6 on every link, so not the
 * unit gauge: otherwise WD_ERR_ARG, and the context holds no gauge field until the
 * next successful call).  The lower-precision copies used by WD_F32/WD_F16/WD_DF32
 * operators are derived from the same field when first needed. */
wd_status wd_set_gauge(wd_ctx *ctx, const double *U_canon, int on_device, int recon);

/* Debug builds (libwd compiled with -DWD_DEBUG; the library's tests build one in
 * paper_1810_04201_gb300/_build_debug/): every neighbour and checkerboard index a
 * Dslash kernel of this context computes is checked against its field, and the first
 * one out of range is kept as 0x80000000 | code << 24 | (index & 0xffffff) (code 1/2:
 * forward/backward neighbour, 3/4: the same on the checkerboard, 5: checkerboard site)
 * while the access goes to index 0 instead.  Writes that word to *word (0: none) and
 * clears it; *is_debug (may be NULL) = 1 for a debug build.  Release builds check
 * nothing and report 0.  No counterpart in the paper: it stands in for a memory
 * checker.  Synchronises the context's stream. */
wd_status wd_debug_word(wd_ctx *ctx, unsigned *word, int *is_debug);

/* Store the links of one precision with another compression than wd_set_gauge's
 * (18, 12 or 8, with the recon = 8 condition above).  No counterpart in the paper: on
 * GB300 the FP64 operator is bound by the FP64 units, so compressed links only add
 * arithmetic there, while the FP32/FP16 operators are bound by memory and gain from
 * them; a mixed-precision solve can keep FP64 links whole (18) and compress the inner
 * precision's (12).  Applies until the next wd_set_gauge, which resets every precision
 * to its recon.  The solvers (wd_cg_solve* and wd_cg_solve_batched) accept any
 * compression for the inner precision when the FP64 links are whole, and otherwise
 * the same compression for both.  Errors: WD_ERR_ARG (bad precision or
 * recon, links unsuited to recon 8), WD_ERR_STATE (no gauge field yet). */
wd_status wd_set_link_compression(wd_ctx *ctx, wd_prec prec, int recon);

/* Bytes of one device field of nrhs right-hand sides in precision prec. */
size_t wd_field_bytes(const wd_ctx *ctx, wd_prec prec, int nrhs);

/* canonical (nrhs x V x 12 complex128, host or device) -> device field. */
wd_status wd_pack(wd_ctx *ctx, const double *canon, int on_device, void *field, wd_prec prec, int nrhs);
/* device field -> canonical (host or device). */
wd_status wd_unpack(wd_ctx *ctx, const void *field, wd_prec prec, int nrhs, double *canon, int on_device);

/* out = D in (section 2.1, Eq. (1)).  in and out are distinct fields of the same
 * precision; gauge precision follows the field precision. */
wd_status wd_apply(wd_ctx *ctx, double kappa, const void *in, void *out, wd_prec prec, int nrhs);
/* out = D^dag in = gamma5 D gamma5 in (section 2.2, gamma5-hermiticity). */
wd_status wd_apply_dagger(wd_ctx *ctx, double kappa, const void *in, void *out, wd_prec prec, int nrhs);
/* out = D^dag D in (section 5: the product the paper moves to hardware).  Uses a
 * context-owned temporary field. */
wd_status wd_normal_apply(wd_ctx *ctx, double kappa, const void *in, void *out, wd_prec prec, int nrhs);

/* out = D^dag D in, like wd_normal_apply, but without allocating device memory.
 *
 * For callers that cannot call cudaMalloc: a process whose device-memory budget is
 * fixed once at start-up (a memory pool that owns the rest of the GPU), or a
 * latency-critical loop that must not pay for cudaMalloc/cudaFree, which may
 * synchronise the whole device.  The paper has no counterpart; this is an
 * interface variant of wd_normal_apply, with the same precisions (WD_F64, WD_F32,
 * WD_F16, WD_DF32) and argument checks (a non-finite kappa is WD_ERR_ARG).
 *
 * The intermediate field D in lives in a fixed file-scope device array of
 * 16 MiB (every GPU that loads the library keeps it until the process exits), so
 * wd_field_bytes(ctx, prec, nrhs) must not exceed 16 MiB: larger requests return
 * WD_ERR_ARG before anything is launched (FP64 fits 16^4 sites with one
 * right-hand side).  The gauge copy of precision prec must already exist, else
 * WD_ERR_STATE: wd_set_gauge creates the WD_F64 copy, the first wd_apply in another
 * precision creates that one, and wd_set_link_compression drops the copy of the
 * precision it changes (WD_F64 included) until the next wd_apply in it.  The
 * context's device must be current.
 *
 * The first call on each context looks up the array's device address
 * (cudaGetSymbolAddress) with the context's device current and keeps it in the
 * context; it is valid in the CUDA context that was current then, like the
 * context's other device buffers.  Make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents; calls whose
 * kernels overlap on the GPU (different streams or host threads) race on it. */
wd_status wd_normal_apply_noalloc(wd_ctx *ctx, double kappa, const void *in, void *out, wd_prec prec, int nrhs);

/* The even-odd Schur operator (FP64): with D = [[1, -kappa H_eo], [-kappa H_oe, 1]] in
 * even/odd blocks (D couples only opposite parities, section 2.1, Eq. (1)), writes
 * (1 - kappa^2 H_eo H_oe) in_e (dagger = 0) or its adjoint (dagger = 1) into the even
 * sites of out and zero into its odd sites.  in, out: WD_F64 fields (one right-hand
 * side, full-lattice layout; the odd sites of in are ignored).  Needs even extents.
 * Uses context-owned half-lattice temporaries. */
wd_status wd_apply_schur(wd_ctx *ctx, double kappa, const void *in, void *out, int dagger);

/* Solver parameters.
 *   tol        stop when ||D^dag(b - D x)|| <= tol ||D^dag b|| (per right-hand side;
 *              see stop_rule)
 *   max_iter   iteration limit
 *   inner_prec WD_F64: plain FP64 CG.  WD_F32 / WD_F16 / WD_DF32: mixed precision --
 *              the Dslash and the inner iteration in FP32 (or FP16 storage with FP32
 *              accumulation, or double-FP32), with FP64 reliable updates
 *              r = D^dag(b - D x) and the solution accumulated in FP64.  WD_F16 (when
 *              the FP32 link copy is compressed as the FP64 or the FP16 copy): between
 *              the FP64 updates, each time the residual has dropped by 1e-2, the
 *              residual is corrected in FP32 from the last FP64 one, r = r64 - A xs
 *              (xs the FP32 partial solution since that update;
 *              wd_cg_result.inner_corrections)
 *   delta      reliable-update trigger: an update runs when the iterated residual
 *              drops below delta times its maximum since the last update (0 = the
 *              default of the inner precision: 3e-6 for WD_F32 and for WD_F16 with
 *              FP32 corrections, 1e-2 for WD_F16 without (3e-3 with precondition =
 *              1), 1e-6 for WD_DF32)
 *   nrhs       number of right-hand sides in b and x (1..WD_MAX_RHS)
 *   block      0: nrhs independent CG recursions sharing each multi-RHS Dslash;
 *              1: block CG (one Krylov space for all right-hand sides, FP64 only)
 *   rhs_tile   right-hand sides per thread block in the solver's multi-RHS Dslash
 *              kernels (0 = the tuned shape; otherwise the tuned site tile, halved
 *              while site tile x rhs_tile exceeds 256; WD_ERR_ARG if that leaves no
 *              block of a multiple of 32 threads)
 *   normal_eq  0: CGNR, D^dag D x = D^dag b (default).  1: CGNE, the form of the
 *              paper's listing (section 2.2): D D^dag y = b from y = 0, then
 *              x = D^dag y; the iterated residual is b - D x itself, tol applies
 *              to ||b - D x|| / ||b||, and the initial guess in x is ignored.
 *              Block CG and the batched solver use CGNR only.
 *   precondition WD_PRECOND_NONE, or WD_PRECOND_EO: even-odd (red-black) Schur
 *              preconditioning.  D couples only sites of opposite parity, so on the
 *              even sites D x = b reduces to (1 - kappa^2 H_eo H_oe) x_e = b_e +
 *              kappa H_eo b_o, solved by CGNR on that operator, with x_o = b_o +
 *              kappa H_oe x_e afterwards.  The reduced system is solved to tol / 2
 *              and resumed from its solution with a tighter tolerance (at most three
 *              times) until the residual stop_rule names, recomputed in FP64 on the
 *              whole lattice, meets tol; iterations are summed.  Needs even extents; CGNR
 *              only (not with block or normal_eq).
 *   stop_rule  WD_STOP_NORMAL (default): tol applies to the normal-equation residual,
 *              ||D^dag(b - D x)|| <= tol ||D^dag b||.  WD_STOP_SYSTEM: tol applies to the
 *              residual of D x = b itself, ||b - D x|| <= tol ||b|| (the residual the
 *              paper's listing iterates, section 2.2), which bounds the solution error by
 *              cond(D) tol.  CGNR iterates the normal residual, so it runs to tol and, while
 *              the recomputed FP64 ||b - D x|| / ||b|| is above tol, resumes from its own
 *              solution with the normal tolerance tightened by the observed ratio of the
 *              two residuals (at most three times; iterations are summed).  With normal_eq
 *              = 1 the iteration already stops on ||b - D x||.  Not with block CG or the
 *              batched solver (WD_ERR_ARG). */
#define WD_PRECOND_NONE 0
#define WD_PRECOND_EO 1
#define WD_STOP_NORMAL 0
#define WD_STOP_SYSTEM 1
typedef struct wd_cg_params {
    double tol;
    int max_iter;
    int inner_prec;
    double delta;
    int nrhs;
    int block;
    int rhs_tile;
    int normal_eq;
    int precondition;
    int stop_rule;
} wd_cg_params;

/* Per right-hand side result.  The two residuals are recomputed from the returned x
 * with the FP64 operator: by a final check after the loop, or, where a mixed-precision
 * solve on the full lattice (or a batched lattice) stopped at a reliable update, by
 * that update, which computed D x and D^dag(b - D x) for the same x. */
typedef struct wd_cg_result {
    int iters;               /* CG iterations */
    int reliable_updates;    /* FP64 residual recomputations (mixed precision) */
    double true_rel_resid;   /* ||D^dag(b - D x)|| / ||D^dag b|| of the returned x, in FP64 */
    double true_rel_resid_b; /* ||b - D x|| / ||b|| of the returned x, in FP64 */
    double seconds;          /* device time of the solve */
    int status;              /* wd_status of this right-hand side */
    int inner_corrections;   /* FP32 corrections of an FP16 inner iteration (wd_cg_solve) */
} wd_cg_result;

/* Solve D x = b for nrhs right-hand sides by CG on D^dag D x = D^dag b, entirely on
 * the device (a CUDA graph with a device-side loop).  b, x: WD_F64 fields of
 * params->nrhs right-hand sides; x holds the initial guess on entry (zeros for the
 * default start; section 2.2, psi <- psi_0) and the solution on exit; for an all-zero
 * guess the setup skips its two operator applications on x (a device-side test).
 * result points to params->nrhs results.  Returns WD_OK when every right-hand side
 * converged. */
wd_status wd_cg_solve(wd_ctx *ctx, double kappa, const void *b, void *x, const wd_cg_params *params,
                      wd_cg_result *result);

/* The same solve on canonical buffers (nrhs x V x 12 complex128) in host memory
 * (on_device = 0; pinned memory gives asynchronous copies) or device memory: packs b
 * and x, solves, unpacks x.  This is the end-to-end call. */
wd_status wd_cg_solve_canonical(wd_ctx *ctx, double kappa, const double *b_canon, double *x_canon, int on_device,
                                const wd_cg_params *params, wd_cg_result *result);

/* Solve n independent lattices, each with its own context (dims, gauge field) and
 * kappa, in one persistent cooperative kernel launch, with mixed-precision
 * (inner_prec) CG and FP64 reliable updates; x[i] holds lattice i's start vector
 * (an all-zero one skips the setup's operator applications on it).  All contexts must live on the same
 * device; the work runs on ctxs[0]'s stream.  b[i], x[i]: WD_F64 fields of ctxs[i]
 * (one right-hand side); result[i] receives lattice i's result.  Every context needs
 * the same pair of link compressions (FP64, inner precision), a pair that
 * wd_set_link_compression's rule allows.  Grid-wide waits
 * inside the kernel are bounded; when one runs out, every result gets
 * WD_ERR_TIMEOUT and the kernel returns. */
wd_status wd_cg_solve_batched(wd_ctx *const *ctxs, const double *kappas, const void *const *b, void *const *x,
                              int n, const wd_cg_params *params, wd_cg_result *result);

/* Autotuner: time the site-tile (threads per block) and right-hand-side-tile
 * choices of the Dslash for this context's lattice, precision and nrhs, and keep
 * the fastest for later calls.  Writes the choice to *site_tile and *rhs_tile
 * (either may be NULL).  Uses context-owned scratch fields; synchronises the stream. */
wd_status wd_autotune(wd_ctx *ctx, wd_prec prec, int nrhs, int *site_tile, int *rhs_tile);
/* Autotuner of the solvers: times the same candidates for the fused CG kernels (the
 * Dslash with the CG epilogues and reductions) as wd_cg_solve runs them -- ten iterations
 * of the device-resident loop in inner precision prec (WD_F64: the plain FP64 solver) on a
 * non-zero right-hand side, L2 flushed before each timed solve -- and keeps the fastest
 * for the solvers of this precision and nrhs (wd_cg_solve, wd_cg_solve_canonical); with all
 * extents even it tunes the even-odd solver's checkerboard kernels too, separately.  The
 * plain operators keep wd_autotune's choice.  *site_tile / *rhs_tile: the choice for plain
 * solves.  Uses and frees context scratch (256 MB for the flush); synchronises the stream. */
wd_status wd_autotune_cg(wd_ctx *ctx, wd_prec prec, int nrhs, int *site_tile, int *rhs_tile);
/* Neighbour staging for the plain FP32 and FP16 operators (the paper's on-chip buffers
 * that feed the stencil pipeline, sections 6.3-6.4): with rows > 0, wd_apply,
 * wd_apply_dagger and wd_normal_apply in precision prec run a persistent kernel whose
 * blocks take tiles of `rows` whole x-rows (rows * Lx sites, rows dividing Ly, at most 256
 * sites) and fetch each tile's neighbour spinors -- the tile, the two adjacent rows, and the
 * same sites one plane and one slice away in each direction, seven contiguous ranges per
 * field array -- into shared memory with 1-D bulk copies completed on an mbarrier, `stages`
 * (2 to 4) tiles in flight per block; links are read directly.  rows = 0 returns to the
 * direct-load kernel (the default; the solvers always use it, since their epilogues are
 * fused into it).  FP16 needs Lx a multiple of 4.  Full lattices only (no split or
 * checkerboard).  Unsupported shapes: WD_ERR_ARG.  No counterpart in the paper beyond the
 * buffers it mirrors. */
wd_status wd_set_staging(wd_ctx *ctx, wd_prec prec, int rows, int stages);
/* Per-thread prefetch for the plain FP32 operator (on = 1): each thread copies the neighbour
 * spinors of its next two hops into its own slots of shared memory with cp.async while it
 * computes the current hop, so more loads are in flight at the same occupancy; links are read
 * directly.  Same launch shapes as the direct kernel (one right-hand side per thread).  No
 * counterpart in the paper beyond the on-chip buffers of sections 6.3-6.4.  on = 0 (default):
 * the direct-load kernel.  Other precisions, split or checkerboard lattices: WD_ERR_ARG. */
wd_status wd_set_prefetch(wd_ctx *ctx, wd_prec prec, int on);
/* The staged kernel bounds its waits; one that ran out since the last call sets *err to 1
 * (and that launch's output is incomplete).  Synchronises the stream and clears the word. */
wd_status wd_staging_error(wd_ctx *ctx, unsigned *err);

/* Fix the tile choice by hand: site_tile in {16, 32, 64, 128, 256} threads,
 * 1 <= rhs_tile <= nrhs, site_tile * rhs_tile <= 256 and a multiple of 32.  WD_F64
 * and WD_DF32 run each site on two lanes (site_tile / 2 sites per block) and need
 * site_tile >= 32.  Unsupported shapes: WD_ERR_ARG. */
wd_status wd_set_tiles(wd_ctx *ctx, wd_prec prec, int nrhs, int site_tile, int rhs_tile);

/* ---- Domain decomposition along t (section 2.3: the lattice is divided into
 * sub-lattices, one per process, each holding copies of its neighbours' boundary sites,
 * and the scalar products of CG are summed over all of them; section 8: multi-node
 * systems).  Rank k of nranks owns the global t-slices [k T / nranks, (k + 1) T / nranks).
 *
 * A split context is the sub-lattice of one rank: Lx x Ly x Lz x (T / nranks) sites,
 * T divisible by nranks, at least one slice each.  Its links and fields use the ordinary
 * layouts of that sub-lattice (wd_set_gauge takes the 4 x V_local x 9 links U_mu(n) of the
 * rank's own sites, the t links of its last slice included; wd_pack / wd_unpack as usual).
 * Its Dslash (WD_F64 or WD_F32, any link compression) is two calls:
 *   wd_apply_interior  every hop whose neighbour is local, with the xpay: out = in - kappa
 *                      (hops); the t hops that leave the sub-lattice are left out;
 *   wd_apply_faces     adds -kappa (the two t hops across the faces) at the first and
 *                      the last slice, from the faces the neighbours sent.
 * wd_face_pack writes the two faces this rank sends, projected half spinors (6 complex
 * numbers per face site, 96 bytes in FP64, 48 in FP32, face site f = x + Lx (y + Ly z)):
 *   to_prev  for rank k - 1 (mod nranks): (1 + s gamma_t) in on the first slice, upper half;
 *   to_next  for rank k + 1 (mod nranks): U_t(n)^dag times the upper half of
 *            (1 - s gamma_t) in on the last slice,
 * with s = -1 for D and +1 for D^dag (dagger).  from_prev of rank k is to_next of rank k - 1,
 * from_next is to_prev of rank k + 1.  With antiperiodic_t the receiver applies the sign of
 * the global boundary (ranks 0 and nranks - 1).  The interior launch does not read the
 * faces, so it can overlap their exchange.  The other operators and solvers refuse split
 * contexts (WD_ERR_STATE). */
wd_status wd_create_split(wd_ctx **ctx, const int global_dims[4], int nranks, int rank, int antiperiodic_t,
                          void *stream);
/* Bytes of one face buffer (nrhs right-hand sides; 0 when ctx is not split or prec is not
 * WD_F64 / WD_F32). */
size_t wd_face_bytes(const wd_ctx *ctx, wd_prec prec, int nrhs);
wd_status wd_face_pack(wd_ctx *ctx, const void *in, void *to_prev, void *to_next, wd_prec prec, int nrhs, int dagger);
wd_status wd_apply_interior(wd_ctx *ctx, double kappa, const void *in, void *out, wd_prec prec, int nrhs, int dagger);
wd_status wd_apply_faces(wd_ctx *ctx, double kappa, const void *from_prev, const void *from_next, void *out,
                         wd_prec prec, int nrhs, int dagger);

/* Communication with the processes that hold the other sub-lattices of a split lattice.
 *   exchange   send send_prev (to_prev of this process's first sub-lattice) to the process
 *              holding the previous rank and receive its to_next into recv_prev; send
 *              send_next (to_next of the last sub-lattice) to the process holding the
 *              next rank and receive its to_prev into recv_next.  Device buffers of `bytes`
 *              bytes; stream is the cudaStream_t the solver works on: the sends may start
 *              after the work queued there, and on return the receive buffers must be
 *              complete in that stream's order.  Returns 0 on success.
 *   allreduce  replace vals[0..n-1] (host memory) by their sums over all processes;
 *              returns 0 on success. */
typedef struct wd_comm {
    void *user;
    int (*exchange)(void *user, const void *send_prev, void *recv_prev, const void *send_next, void *recv_next,
                    size_t bytes, void *stream);
    int (*allreduce)(void *user, double *vals, int n);
} wd_comm;

/* CGNR (section 2.2) on a lattice split along t: ctxs[0..n-1] are the sub-lattices this
 * process holds, consecutive ranks on one device (all of them when n = nranks, and then
 * comm may be NULL); b[i], x[i] their WD_F64 fields (x: start vector in, solution out).
 * Faces between local sub-lattices are exchanged by device copies on a side stream while
 * the interior launches run; faces to other processes and every scalar product go through
 * comm.  Each iteration sums |D p|^2 and |r|^2 over all sub-lattices, and the host takes
 * alpha, beta and the stopping test (the division of labour of the paper's section 5).
 * params: plain FP64 (inner_prec WD_F64), nrhs 1, no block, CGNE, preconditioner or
 * system stopping rule (WD_ERR_ARG otherwise); tol applies to the normal residual.
 * *result (one, for the whole lattice) holds the residuals of the returned x recomputed
 * on the whole lattice; the work runs on ctxs[0]'s stream and the call waits for it. */
wd_status wd_cg_solve_split(wd_ctx *const *ctxs, int n, double kappa, const void *const *b, void *const *x,
                            const wd_cg_params *params, wd_cg_result *result, const wd_comm *comm);

/* Measured FP64 arithmetic rate of the current device, in GFLOP/s (2 flop per fused
 * multiply-add): independent FP64 multiply-add chains on every SM, no memory traffic,
 * timed with CUDA events on a stream of its own (best of five launches after one
 * warm-up).  No counterpart in the paper: on GB300 the FP64 Dslash is bound by the
 * FP64 units, and this is the roof it is reported against.  Synchronises that stream;
 * changes no device setting.  Errors: WD_ERR_ARG (null), WD_ERR_CUDA. */
wd_status wd_measure_fp64_rate(double *gflops);

/* The launch shape the plain operators of (prec, nrhs) use now: site_tile, rhs_tile and
 * rhs_per_thread (any pointer may be NULL). */
wd_status wd_get_tiles(wd_ctx *ctx, wd_prec prec, int nrhs, int *site_tile, int *rhs_tile, int *rhs_per_thread);
/* Plain FP32 operators: each thread applies its site's links to k (1 to 4) of its block's
 * right-hand sides, loading each link once for all k (k dividing rhs_tile, and
 * site_tile * rhs_tile / k threads a multiple of 32); wd_autotune considers k = 2, 3, 4
 * beside 1.  Other precisions, the solvers' fused kernels and split sub-lattices
 * (WD_ERR_STATE for k > 1): k = 1 only.  No counterpart in the paper, which has one
 * right-hand side. */
wd_status wd_set_rhs_per_thread(wd_ctx *ctx, wd_prec prec, int nrhs, int k);

/* Launch-configuration query: number of kernel launches the last wd_* call queued
 * (graph kernel nodes count once per execution). */
long long wd_kernel_launches(const wd_ctx *ctx);

const char *wd_status_string(wd_status s);
const char *wd_last_error(const wd_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* WD_H */

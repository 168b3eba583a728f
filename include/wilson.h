/*
 * wilson.h -- C ABI of the GB300 (sm_103a) Wilson-fermion multi-mass solver.
 *
 * Method: Alexandru, Pelissier, Gamari & Lee, "Multi-mass solvers for lattice
 * QCD on GPUs" (arXiv:1103.5103).  The library solves M(m_i) x_i = b for
 * several bare masses m_i with the Wilson-Dirac operator
 *     M_p(m) = (m + 4) - D/2                                 (Eq. 3)
 *     (D psi)_n = sum_mu [ U_mu(n) psi_{n+mu} (1 - gamma_mu)
 *                        + U_mu(n-mu)^dag psi_{n-mu} (1 + gamma_mu) ]  (Eq. 4)
 * where psi_n is a 3x4 matrix (colour rows, spin columns) and the spin matrix
 * multiplies from the right, with the gamma matrices of Section 2.  The
 * library works in the kappa normalisation
 *     M_k = 1 - kappa D,  kappa = 1 / (2 m0 + 8),   M_p = (m0 + 4) M_k,
 * so a solution x of M_k x = b is (m0 + 4) times the paper's psi; relative
 * residuals are identical in both normalisations.  Hops across the time
 * boundary carry -1 when the lattice is antiperiodic in time; space is
 * periodic.
 *
 * Conventions for every call
 *  - Returns an int status (WL_OK = 0); wl_last_error() gives a thread-local
 *    message for the last failing call on this thread.  No C++ exception
 *    crosses this interface.
 *  - "stream" is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - Field arrays are caller-owned DEVICE pointers; the library never frees
 *    them.  The canonical sources and solutions of the solvers and of
 *    wilson_dslash may instead be page-locked HOST memory (cudaHostAlloc or
 *    cudaHostRegister): with unified addressing the layout kernels read and
 *    write it directly over the host link, so no separate copy is needed.
 *    Handles (wl_lattice, wl_gauge) are library-owned: the caller
 *    destroys them.  A wl_gauge also owns the solver workspace, allocated on
 *    first use with cudaMalloc and released by wl_gauge_destroy.
 *  - Canonical external layout (complex128, interleaved re/im):
 *      site index  n = x + X*(y + Y*(z + Z*t))
 *      spinor      [n][spin 4][colour 3]                (12 complex per site)
 *      links       [mu 4][n][row 3][col 3], mu = 0..3 <-> x, y, z, t
 *                  (the paper's gamma_1..gamma_4 directions)
 *    Sources and solutions are full-lattice vectors; the even/odd split is
 *    internal.  Site parity = (x+y+z+t) mod 2; site 0 is even.
 *  - Precisions: WL_F64, WL_F32, WL_F16 (FP16 storage with one FP32 norm
 *    per site, arithmetic in FP32) and WL_DF (double-float, see below).
 *    FP32 links are stored as their first two rows (12 reals) and the third
 *    row is rebuilt as conj(row0 x row1), which is exact for SU(3) links;
 *    FP64 and FP16 links keep all three rows as given and double-float links
 *    all three rows with row 2 formed in FP64 when the handle is created.
 */
#ifndef WILSON_H
#define WILSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define WL_OK            0
#define WL_ERR_ARG       1  /* bad dims, odd extent, NULL pointer, duplicate masses, bad enum */
#define WL_ERR_CUDA      2  /* a CUDA runtime call failed                                    */
#define WL_ERR_OOM       3  /* device allocation failed                                      */
#define WL_ERR_NOCONV    4  /* iteration cap reached; outputs hold the last iterate           */
#define WL_ERR_BREAKDOWN 5  /* Krylov breakdown that restarts could not cure                  */
#define WL_ERR_TIMEOUT   6  /* a bounded device wait ran out                                  */
#define WL_ERR_CHECKED   7  /* reserved for a bounds-checked build (a recorded index
                               violation); no call of this library returns it            */

/* ------------------------------------------------------------- precisions */
#define WL_F64 1
#define WL_F32 2
#define WL_F16 4
#define WL_DF  8  /* double-float: a value is hi + lo of two FP32 numbers (about 48
                     significant bits); arithmetic by error-free transformations on
                     the FP32 pipes.  Used for the outer (reliable-update) loop. */

/* ----------------------------------------------------------------- parity */
#define WL_EVEN 0
#define WL_ODD  1

/* ----------------------------------------------------- dslash operator ids */
#define WL_OP_HOP   0  /* out = D in                        (full lattice)     */
#define WL_OP_M     1  /* out = in - kappa D in             (full lattice)     */
#define WL_OP_MPREC 2  /* out_e = in_e - kappa^2 D_eo D_oe in_e, out_o = 0     */

/* ------------------------------------------------------ solver parameters */
#define WL_GUESS_ZERO 0  /* zero initial guess for every mass                     */
#define WL_GUESS_POLY 1  /* Lagrange extrapolation through the previous masses
                            (Section 6.2.1, Eq. Poly)                           */
#define WL_GUESS_SSM  2  /* solution-space minimisation: the combination of the
                            previous solutions with the smallest residual
                            (Section 6.2.2)                                     */
#define WL_SOLVER_BICGSTAB 0  /* inner Krylov solver: BiCGstab on M_prec (the paper's)     */
#define WL_SOLVER_CG       1  /* CG on the normal equations M_prec^dag M_prec e = M_prec^dag r
                                 (Section 8 expects the findings to carry over to CG); the
                                 inner stop is on the true inner residual r - M_prec e      */

#define WL_MODE_HOST       0  /* one host round trip per iteration                      */
#define WL_MODE_GRAPH      1  /* iterations captured in a CUDA graph, scalars on device */
#define WL_MODE_PERSISTENT 2  /* one cooperative kernel runs whole iterations; phases
                                 separated by grid barriers with a bounded wait        */

typedef struct wl_lattice wl_lattice;
typedef struct wl_gauge wl_gauge;

typedef struct {
    double tol;          /* target true relative residual ||b - M x|| / ||b||        */
    int    max_iter;     /* cap on Krylov iterations per mass (all restarts)          */
    int    inner_prec;   /* WL_F64, WL_F32 or WL_F16: precision of the Krylov loop    */
    double inner_tol;    /* defect-correction inner relative tolerance; 0 = default   */
    int    max_restarts; /* cap on outer FP64 restarts per mass                        */
    int    guess;        /* WL_GUESS_*  (multimass_solve)                              */
    int    mode;         /* WL_MODE_*                                                   */
    int    rhs_block;    /* right-hand sides per thread in batched hops; 0 = autotune  */
    int    graph_iters;  /* iterations per captured graph (WL_MODE_GRAPH)               */
    int    eo;           /* 1: even-odd preconditioned solve (bicgstab_solve)           */
    int    outer_prec;   /* WL_F64 or WL_DF: precision of the residual recomputation
                            b - M x, of the solution accumulator and of the even-odd
                            reconstruction                                           */
    const void *shadow;  /* bicgstab_m_solve only: the shadow residual rhat of the
                            BiCGstab recurrences, a canonical complex128 full-lattice
                            device vector owned by the caller, or NULL for rhat = b.
                            With rhat = b a point source, <rhat, r_1> vanishes after
                            one iteration (closed two-hop paths are backtracks and
                            (1 - gamma_mu)(1 + gamma_mu) = 0), so point sources need
                            a shadow such as Gaussian noise.  <rhat, b> must not
                            vanish (WL_ERR_ARG).                                      */
    int    guess_max;    /* multimass_solve: previous masses the guess uses, the most
                            recently solved (nearest) ones; 0 = all of them.  With
                            a limit the solver keeps only guess_max + 1 stored
                            solutions per source (a ring), not one per mass      */
    int    reliable;     /* mixed-precision outer loop: 0 = restarted defect
                            correction (Section 6.2.4: each outer step restarts the
                            inner BiCGstab on the FP64-class residual); 1 = reliable
                            updates (the method the paper cites there): the inner
                            BiCGstab keeps its shadow residual and search direction,
                            and only r is replaced by the true residual and the
                            correction folded into x when the inner residual has
                            dropped by inner_tol                                      */
    int    inner_solver; /* WL_SOLVER_BICGSTAB (default) or WL_SOLVER_CG; CG works with
                            the graph and host modes and restarted defect correction  */
    int    verify_full;  /* even-odd solves: how stats.true_relres gets the even half of
                            the full-lattice residual.  0 (default): from the last
                            outer check, b_prec - M_prec x_e, which equals
                            b_e - x_e + kappa D_eo x_o up to the rounding of the
                            rebuilt x_o = b_o + kappa D_oe x_e (Section 6.2.3), so no
                            further hop; 1: recomputed with one more outer-precision
                            hop D_eo x_o per rhs.  The odd half is the rounding of
                            the rebuild either way.                                  */
    int    outer_blocks_per_sm; /* FP64 outer loop: 0 (default) launches the residual
                            hops with the autotuned full grid; 1 or 2 launches them as
                            a grid-stride kernel of that many 128-thread blocks per SM.
                            The FP64 hop is bound by the FP64 pipe and needs few warps;
                            the small grid leaves the rest of each SM to work on other
                            streams, such as the inner solve of another batch of
                            sources solved at the same time on another handle.      */
    int    inner_refine; /* FP16 BiCGstab inner solves without reliable updates: 1
                            runs each outer step's inner solve as FP16 segments with
                            the inner residual recomputed in FP32 between them, so
                            that one outer step reaches inner_tol (default 1e-7) of
                            its residual instead of the FP16 limit near 3e-4 and the
                            solve needs fewer outer (FP64) residual checks.  An outer
                            step whose target lies above the FP16 limit runs one
                            segment, unchecked in FP32.  The handle then needs FP32
                            links (else WL_ERR_ARG).  Other inner solves ignore it.
                            0 (default): one FP16 solve per outer step.              */
} wl_solver_params;

typedef struct {
    double mass;         /* bare mass m0 of this solve                                 */
    int    status;       /* WL_OK, WL_ERR_NOCONV or WL_ERR_BREAKDOWN                    */
    int    iterations;   /* Krylov iterations (sum over restarts)                       */
    int    matvecs;      /* applications of the solved operator                         */
    int    restarts;     /* outer FP64 restarts (defect-correction steps)               */
    double true_relres;  /* FP64 ||b - M_k x|| / ||b|| on the full lattice at exit      */
    double seconds;      /* wall time of this mass's solve (host clock, stream synced)  */
} wl_solver_stats;

/* Fill *p with defaults: tol 1e-10, max_iter 100000, inner WL_F32,
 * inner_tol 0 (1e-6 for FP32, 3e-4 for FP16, 1e-12 for FP64; never below
 * what the outer target needs), max_restarts 100,
 * WL_GUESS_POLY, WL_MODE_GRAPH, rhs_block 0, graph_iters 8, eo 1,
 * outer_prec WL_F64, shadow NULL, guess_max 0, reliable 0,
 * inner_solver WL_SOLVER_BICGSTAB, verify_full 0, outer_blocks_per_sm 0,
 * inner_refine 0. */
int wl_params_default(wl_solver_params *p);

/* Thread-local message describing the last failing call on this thread. */
const char *wl_last_error(void);

/* --------------------------------------------------------------- geometry */

/* Create a lattice of extents dims = {X, Y, Z, T}.  Every extent must be even
 * and >= 2 (the even/odd split of Section 6.2.3 needs it) and the volume
 * below 2^31.  antiperiodic_t: 1 gives -1 on hops across the time boundary.
 * Host-only; no device work. */
int wl_lattice_create(const int dims[4], int antiperiodic_t, wl_lattice **out);
int wl_lattice_destroy(wl_lattice *lat);

/* Bytes of one internal half-lattice (one parity) spinor of precision prec.
 * Internal spinors are site-blocked structure-of-arrays per parity
 * (Section 4, Eq. 7, re-laid for 128-bit loads). */
int wl_spinor_bytes(const wl_lattice *lat, int prec, size_t *bytes);

/* Convert one parity of a canonical full-lattice complex128 spinor (device)
 * to the internal format of precision prec (device, wl_spinor_bytes bytes),
 * and back.  Export writes only the sites of the given parity. */
int wl_spinor_import(const wl_lattice *lat, const void *canon_c128, void *internal, int prec,
                     int parity, void *stream);
int wl_spinor_export(const wl_lattice *lat, const void *internal, void *canon_c128, int prec,
                     int parity, void *stream);

/* Pack canonical complex128 links (device, [4][V][3][3]) into the internal
 * per-parity layouts (Section 4, Eq. 8; FP32 compressed to two rows, FP64,
 * FP16 and double-float with all three) for every precision set in
 * prec_mask (WL_F64 | WL_F32 | WL_F16 | WL_DF).  The links must be SU(3):
 * the FP32 format and the TMA-staged FP16 hop rebuild the third row from
 * the first two.  Links whose U U^dag - 1 or det U - 1 has an entry (real or
 * imaginary part) above 1e-6 in magnitude, or a NaN, are rejected with
 * WL_ERR_ARG.  The gauge handle keeps a reference to lat, which must
 * outlive it.  Synchronises the stream before returning. */
int wl_gauge_create(wl_lattice *lat, const void *U_canon_c128, unsigned prec_mask, void *stream,
                    wl_gauge **out);
int wl_gauge_destroy(wl_gauge *g);

/* ---------------------------------------------------------------- dslash */

/* One parity hop on internal spinors (Section 2, Eq. 4; Algorithm 1 without
 * the diagonal term):  out = x + coef * D_{p,1-p} in,  or out = coef * D in
 * when x is NULL.  out_parity p selects D_eo (p = WL_EVEN) or D_oe.
 * dagger = 1 applies D^dag = gamma5 D gamma5.  in, x, out are internal
 * spinors of precision prec (in has the other parity); out must not alias
 * in.  The gauge handle must hold links of precision prec. */
int wilson_hop(wl_gauge *g, const void *in, void *out, const void *x, double coef, int prec,
               int out_parity, int dagger, void *stream);

/* Batched hop over n_rhs internal spinors of one parity laid out rhs_stride
 * bytes apart (rhs_stride >= wl_spinor_bytes, a multiple of 256):
 *   out_r = x_r + coef * D_{p,1-p} in_r   (x may be NULL: out_r = coef D in_r).
 * Thread blocks are ordered with the rhs index fastest, so the blocks that
 * read a given link run together and the link comes from HBM once per
 * launch; rhs_block (1, 2 or 4) rhs are handled by one thread, which then
 * loads each link into registers once for all of them; rhs_block = 0 uses
 * the variant chosen by wl_autotune for (prec, n_rhs), or 1 if untuned; a
 * negative rhs_block selects the autotuner variant -rhs_block directly. */
int wilson_hop_multi(wl_gauge *g, const void *in, void *out, const void *x, double coef, int prec,
                     int out_parity, int dagger, int n_rhs, size_t rhs_stride, int rhs_block, void *stream);

/* Canonical full-lattice operator application (complex128 in and out):
 *   WL_OP_HOP   out = D in
 *   WL_OP_M     out = in - kappa D in                        (Eq. 3, kappa form)
 *   WL_OP_MPREC out_e = in_e - kappa^2 D_eo D_oe in_e, out_o = 0   (Eq. eo4)
 * computed in precision prec through the internal layout.  Scratch comes
 * from the gauge handle's workspace.  in and out must not alias. */
int wilson_dslash(wl_gauge *g, const void *in, void *out, double kappa, int prec, int op,
                  void *stream);
/* The adjoint of the same operator: D^dag = gamma5 D gamma5. */
int wilson_dslash_dag(wl_gauge *g, const void *in, void *out, double kappa, int prec, int op,
                      void *stream);

/* The same operator application as wilson_dslash / wilson_dslash_dag
 * (dagger = 0 / 1), for callers that must not allocate device memory: code
 * running while another component owns the allocator (a caching allocator
 * with a hard cap, a pool that must not fragment, a loop that cannot take
 * cudaMalloc's implicit synchronisation).  The paper has no counterpart.
 * wilson_dslash takes four internal half-lattice spinors from the gauge
 * handle's workspace and allocates it on first use; this entry point takes
 * them from a fixed 64 MiB array compiled into the library (held by every
 * GPU that loads the library until the process exits) and calls no
 * cudaMalloc, cudaFree or allocating routine.  Lattices whose four
 * half-lattice spinors of precision prec exceed 64 MiB are rejected with
 * WL_ERR_ARG.  The first call on a device looks up the array's device
 * address (with lazy module loading this also makes the driver load the
 * library's module); make that first call before any stream capture.  The
 * address is cached per device and is stale after cudaDeviceReset: do not
 * call it after a device reset.  All calls share the array: calls whose work
 * overlaps on the GPU (different streams or threads) race on it -- order
 * them on one stream.  The call holds the handle's lock, like every other
 * call on a wl_gauge. */
int wilson_dslash_noalloc(wl_gauge *g, const void *in, void *out, double kappa, int prec, int op, int dagger,
                          void *stream);

/* --------------------------------------------------------------- solvers */

/* Solve M_k(m0) x = b (Section 6) with BiCGstab.  b, x: canonical
 * full-lattice complex128 device vectors; x holds the initial guess on entry
 * and the solution on exit.  With p->eo = 1 the even-odd preconditioned
 * system M_prec x_e = b_e + kappa D_eo b_o is solved and x_o is rebuilt
 * (Section 6.2.3); with p->inner_prec below FP64 each outer step recomputes
 * the FP64 residual and runs a reduced-precision inner BiCGstab
 * (defect correction, Section 6.2.4).  Stops when the FP64 preconditioned
 * residual is below tol * ||b||; stats->true_relres is the FP64 full-lattice
 * residual of the returned x.  Synchronises the stream.
 * Returns WL_OK, WL_ERR_NOCONV or WL_ERR_BREAKDOWN (x = best iterate). */
int bicgstab_solve(wl_gauge *g, const void *b, void *x, double m0, const wl_solver_params *p,
                   wl_solver_stats *stats, void *stream);

/* Multi-shift BiCGstab-M baseline (Section 6.1): one Krylov space built on
 * the full-lattice unshifted system M_p(m_s), m_s = min m0[i], shifts
 * sigma_i = m0[i] - m_s, converged shifts frozen, loop ends when the
 * unshifted residual is below tol * ||b||.  No even-odd preconditioning
 * (the paper: multi-shift cannot use it) and no reduced precision (the
 * shifted recurrences need the full Krylov space): the vectors and hops run
 * in p->outer_prec, WL_F64 (needs FP64 links) or WL_DF (double-float, needs
 * double-float links); inner_prec is not used.  x[i] receives the
 * kappa-form solution (m0[i] + 4) psi_i as a canonical complex128 vector.
 * A shift whose true residual is still above tol afterwards is polished by
 * a single-mass BiCGstab from x[i] (FP64 inner where the handle has FP64
 * links, else FP32 inner and outer_prec outer, which needs FP32 links: a
 * polish that finds neither returns WL_ERR_ARG in stats[i].status); its
 * extra iterations are counted in stats[i].restarts.  The shadow residual is p->shadow (NULL: b).
 * Returns WL_ERR_BREAKDOWN, with the polished solutions in x, when the
 * shifted recurrences broke down.  Masses must be distinct.  Synchronises
 * the stream. */
int bicgstab_m_solve(wl_gauge *g, const void *b, void *const *x, const double *m0, int n_mass,
                     const wl_solver_params *p, wl_solver_stats *stats, void *stream);

/* The paper's single-mass multi-mass scheme (Sections 6.2 and 7): masses
 * sorted heaviest first; each solved with even-odd preconditioned,
 * mixed-precision BiCGstab; initial guess for mass k by Lagrange
 * extrapolation through all k-1 previous solutions (Eq. Poly, extrapolating
 * the paper-normalised psi = x / (m0 + 4)), or, with p->guess =
 * WL_GUESS_SSM, by the combination of them with the smallest residual
 * (Section 6.2.2; the Gram matrix of the solutions is formed on the
 * canonical outputs x as they are written, and the k x k normal equations
 * are solved on the host); p->guess_max limits either to the most recent
 * solutions.  The first residual of each mass is the same linear
 * combination of the stored D_eo D_oe x_j, so it costs no hop; a hop-based
 * check confirms convergence.  b[r] (r < n_rhs) are canonical
 * sources; x[r * n_mass + i] receives the solution for source r and mass
 * m0[i]; stats[r * n_mass + i] its statistics.  All right-hand sides of one
 * mass are solved together by batched kernels.  The solutions of a
 * finished mass are written to x on an internal stream while the next mass
 * is solved; every write is complete when the call returns.  Masses must be
 * distinct.  Synchronises the stream. */
int multimass_solve(wl_gauge *g, const void *const *b, void *const *x, int n_rhs, const double *m0,
                    int n_mass, const wl_solver_params *p, wl_solver_stats *stats, void *stream);

/* Backward of the multi-mass solve (gradient of a real loss L(x_1..x_n),
 * x_i = M_k(m0[i])^{-1} b, Eq. 3-4 in kappa form).  g[i] is the loss
 * gradient with respect to x_i in PyTorch's complex convention,
 * dL/dRe x + i dL/dIm x (canonical complex128, device).  For each mass the
 * adjoint system M_k^dag lam = g[i] is solved through M^dag = gamma5 M gamma5
 * (lam = gamma5 M^{-1} gamma5 g, the forward solver with parameters p), then
 *   dU  [mu][n][a] += -kappa Im tr(T_a W_mu(n)),  T_a = lambda_a / 2,
 *        W_mu(n) = s [U_mu(n) x_{n+mu} (1 - gamma_mu) lam_n^dag
 *                     - x_n (1 + gamma_mu) lam_{n+mu}^dag U_mu(n)^dag],
 *        s = -1 across the antiperiodic time boundary: the derivative along
 *        U_mu(n) -> exp(i h T_a) U_mu(n) at h = 0 (device doubles [4][V][8],
 *        accumulated: the caller zeroes them);
 *   dm0 [i] = -Re <lam, 2 kappa^2 D x_i>   (host doubles, n_mass);
 *   db      += lam                           (device complex128, optional).
 * x[i] may be NULL (or x itself NULL): that solution is re-solved instead of
 * stored.  Any of dU, dm0, db may be NULL (not computed).  Needs FP64 or
 * double-float links.  Synchronises the stream. */
int wilson_solve_backward(wl_gauge *g, const void *b, const void *const *x, const void *const *g_x,
                          const double *m0, int n_mass, const wl_solver_params *p, double *dU, double *dm0,
                          void *db, void *stream);

/* ------------------------------------------------------------ profiling */

/* Live timing of the dominant kernel, the hop D_oe p that opens every inner
 * BiCGstab iteration.  While profiling is on, each iteration records a pair
 * of CUDA events around that launch on the solve's stream (inside the
 * captured graph in WL_MODE_GRAPH); the solver adds up their elapsed times
 * at the host synchronisation that already follows every block of
 * iterations.  Only iterations in which every right-hand side was still
 * active are counted, so each counted launch processed exactly
 * n_rhs * V/2 output sites. */
typedef struct {
    long long launches;    /* counted hop launches                               */
    double    ms;          /* summed CUDA-event durations of those launches      */
    double    site_rhs;    /* sum over counted launches of (V/2) * n_rhs          */
    double    sites;       /* sum over counted launches of V/2 (link-reuse model) */
} wl_kernel_profile;

/* Reset the counters of g and start (on = 1) or stop (on = 0) profiling. */
int wl_profile_enable(wl_gauge *g, int on);
/* Counters of the inner hop per inner precision: out[0] FP64, out[1] FP32,
 * out[2] FP16; out[3]: the outer loop's residual hop D_oe x that opens every
 * defect-correction check (outer precision), timed the same way, with
 * site_rhs counting only the rhs that the launch processed. */
int wl_profile_read(wl_gauge *g, wl_kernel_profile out[4]);

/* Autotune the hop for (prec, n_rhs) on this gauge handle: every variant
 * (right-hand sides per thread, minimum resident blocks per SM) is timed
 * with CUDA events on the stream and the fastest is cached in the handle;
 * solvers and wilson_hop_multi with rhs_block = 0 use it.  With the
 * environment variable WL_AUTOTUNE_CACHE naming a file, results are read
 * from and appended to it.  *variant = 100 * rhs-per-thread + min-blocks,
 * *best_us its time per launch.  Synchronises the stream. */
int wl_autotune(wl_gauge *g, int prec, int n_rhs, void *stream, int *variant, double *best_us);

/* Number of bounded waits that gave up on the device since the last reset
 * (no paper counterpart).  The TMA-staged hop variants wait on an mbarrier
 * for each tile's copies; a wait that does not complete within about a
 * second of clock cycles is counted here, and that block stops instead of
 * hanging.  Reads the counter into *count after synchronising the stream
 * and, with reset = 1, sets it back to zero.  Autotuning and the inner
 * solver check it and return WL_ERR_TIMEOUT when it is non-zero. */
int wl_wait_faults(unsigned *count, int reset, void *stream);

/* One fused vector kernel of the BiCGstab iteration (Section 5: the vector
 * utilities, here one pass per update with its reductions) applied to
 * caller-owned internal half-lattice vectors: n_rhs vectors of precision
 * prec (WL_F64, WL_F32 or WL_F16; the layout wl_spinor_import writes),
 * rhs_stride bytes apart (a multiple of 256), vecs[k] the first rhs of
 * operand k.  Per-rhs complex scalars in scal[6 r .. 6 r + 5] = alpha,
 * omega, beta (re, im each).  A test hook for the kernels the solvers run:
 *   WL_VEC_S      s = r - alpha v                          vecs r, v, s
 *   WL_VEC_XR     x += alpha p + omega s; r = s - omega t  vecs x, p, s, t, r, rhat
 *                 (x is FP32 for FP32 and FP16 data, FP64 for FP64);
 *                 dots[3 r ..]: <rhat, r> (re, im) and ||r||^2 of the new r
 *   WL_VEC_P      p = r + beta (p - omega v)               vecs r, p, v
 *   WL_VEC_NORM2  dots[r] = ||a||^2                        vecs a
 * Inner products: FP32 per site, FP32 within a warp, FP64 across warps and
 * blocks.  Synchronises the stream. */
#define WL_VEC_S     0
#define WL_VEC_XR    1
#define WL_VEC_P     2
#define WL_VEC_NORM2 3
int wl_vector_op(wl_gauge *g, int kind, int prec, int n_rhs, size_t rhs_stride, void *const *vecs,
                 const double *scal, double *dots, void *stream);

/* Bounds-checked build (no paper counterpart): libwilson_checked.so is the
 * same library compiled with every site index of an internal spinor or link
 * access tested against its array length.  The first violation in each
 * translation unit is recorded and the access is redirected to site 0 (a
 * load) or dropped (a store); nothing traps.  Synchronising calls
 * (multimass_solve, bicgstab_solve, bicgstab_m_solve,
 * wilson_solve_backward, and in this build wilson_dslash,
 * wilson_dslash_dag, wilson_hop, wilson_hop_multi) then return
 * WL_ERR_CHECKED.  wl_checked_status synchronises the device and writes the
 * first recorded violation to *first (0: none; otherwise bit 63 set, the
 * access kind -- 1 spinor load, 2 spinor store, 3 link load -- in bits
 * 32-39 and the site index in bits 0-31), clearing the records if reset
 * is 1.  In the ordinary library *first is always 0.
 * wl_is_checked_build returns 1 in the checked library, 0 otherwise. */
int wl_checked_status(unsigned long long *first, int reset);
int wl_is_checked_build(void);

/* Failure-path check of the persistent solver (WL_MODE_PERSISTENT): runs
 * one cooperative launch of the persistent BiCGstab on zero vectors with
 * the barrier wait limited to wait_limit_s seconds.  With
 * inject_missing_arrival = 1 one block skips its first barrier arrival, so
 * every other block's bounded wait runs out: the kernel exits and the call
 * returns WL_ERR_TIMEOUT while the context stays usable.  With 0 it returns
 * WL_OK.  The paper has no counterpart (it concerns this library's own
 * barrier).  Synchronises the stream. */
int wl_persistent_selftest(wl_gauge *g, int prec, int inject_missing_arrival, double wait_limit_s, void *stream);

/* Number of kernels this library has launched in the process so far (direct
 * launches plus, for every replay of a captured graph, its kernel nodes). */
int wl_launch_count(long long *out);

#ifdef __cplusplus
}
#endif

#endif /* WILSON_H */

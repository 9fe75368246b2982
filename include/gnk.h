/*
 * gnk.h -- C ABI of libgnk: GB300 (sm_103a) Nystrom solver for the boundary
 * integral equations with the generalized Neumann kernel (Nasser, "Fast
 * solution of boundary integral equations with the generalized Neumann
 * kernel").
 *
 * Problem statement (Sec. 1): for an (m+1)-connected domain G with boundary
 * parametrisation eta(t) on the (m+1) n trapezoidal nodes t_{kn+p} = (p-1)2pi/n
 * (Eq. ti-skp, component-major), coefficient A(t) of Eq. (A) and data gamma,
 *   (I - N) mu = -M gamma,  h = [M mu - (I - N) gamma] / 2     (Eqs. ie, h)
 *   (I + N* + J) mu = gamma                                   (Eq. ie*)
 * discretised with singularity subtraction as (Eqs. sys, y, bh, sys*)
 *   (2I + diag(B1) - B) mu = -y,  y = (D - diag(D1) + Lhat) gamma,
 *   (diag(e) + B^T + Phat) mu = gamma.
 * Every product with B, D, B^T and e reduces to the Cauchy sum
 *   (E w)_i = sum_{j != i} w_j / (eta_i - eta_j)              (Eq. fmm-E)
 * which this library evaluates on the GPU either as a direct all-pairs sum
 * (FP64, FP32 or double-float) or by the fast multipole method (Sec. 2.5,
 * the paper's own route), chosen per call by a GNK_PREC_* precision.
 *
 * Conventions for every function below:
 *   - Return value: GNK_OK (0) or a negative GNK_E* code; gnk_last_error()
 *     returns the message of the calling thread's last failure.
 *   - Complex arrays are interleaved (re, im) doubles: length 2*N doubles for
 *     N = (m+1) n nodes.  Real arrays are N doubles.
 *   - Pointers may be device memory or host memory; the library checks which
 *     (cudaPointerGetAttributes).  Host arrays are staged through device
 *     buffers owned by the boundary handle; a call that writes to a host
 *     array returns after the data has arrived (it synchronises `stream`).
 *     Device outputs are written asynchronously on `stream`.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     on one handle must not overlap: the handle's workspace is shared.
 *   - Argument checks (sizes, NULL pointers, n even) happen before any launch
 *     and return GNK_EINVAL.  CUDA failures return GNK_ECUDA, and so does a
 *     solve in which a kernel's bounded wait gave up (the Arnoldi step's grid
 *     barriers and bulk copies, the FMM near field's copy pipeline: no wait
 *     spins without a limit); the message says which.
 *   - GMRES orthogonalises in double-float (about 48 significant bits) for
 *     every precision but GNK_PREC_FP64, which keeps it in FP64.
 *   - The caller owns all arrays it passes; the handle owns its own copies.
 */
#ifndef GNK_H
#define GNK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GNK_OK          0
#define GNK_EINVAL     -1  /* bad argument: sizes, NULL pointer, odd n, ...     */
#define GNK_ENOTCONV   -2  /* solver stopped at maxit; best iterate written       */
#define GNK_ENONFINITE -3  /* NaN/Inf met in the input or in the iteration        */
#define GNK_ECUDA      -4  /* CUDA runtime error                                  */
#define GNK_ENOMEM     -5  /* device allocation failed                            */

/* Arithmetic of the pair sums (the Cauchy sums E w). */
#define GNK_PREC_FP64  0   /* FP64 pair sums everywhere                           */
#define GNK_PREC_MIXED 1   /* FP32 pair sums inside GMRES, wrapped in FP64
                              iterative refinement (residual, circulant part,
                              diagonals and Givens rotations stay FP64)          */
#define GNK_PREC_FP32  2   /* FP32 pair sums (apply/cauchy calls only)            */
#define GNK_PREC_DF32  3   /* double-float pair sums: pairs of FP32 values carried
                              through error-free transformations on the FP32
                              pipe, about 2^-46 relative per term (FP64-class
                              accuracy; GB300's FP64 pipe is 1/64 of FP32)     */
#define GNK_PREC_MIXED_DF 4 /* as GNK_PREC_MIXED, with the refinement residual,
                              right-hand side and h in double-float pair sums  */
#define GNK_PREC_FMM   5   /* Cauchy sums by the fast multipole method (Sec. 2.5:
                              the paper's zfmm2dpart route), FP64, expansion
                              order 32: error below ~1e-12 of
                              sum_j |w_j / (eta_i - eta_j)|, O(N) work.  The
                              quadtree is built on the first such call (on the
                              device; on the host when it is deeper than 11
                              levels) and kept with the handle, whose FMM
                              workspace also serialises its products: one
                              handle is not used on two streams at once.     */
#define GNK_PREC_MIXED_FMM 6 /* as GNK_PREC_MIXED, with the refinement residual,
                              right-hand side and h by the FMM               */

typedef struct gnk_boundary gnk_boundary;

/* GMRES controls, with the meaning of MATLAB's gmres(restart, tol, maxit)
 * used by the paper (Sec. 3.5, Eq. ie-gmres): x0 = 0, no preconditioner,
 * `restart` inner iterations per cycle, at most `maxit` cycles, stop when
 * ||b - A x||_2 / ||b||_2 <= tol. */
typedef struct gnk_options {
    int restart;       /* inner iterations per cycle (>= 1)                    */
    int maxit;         /* maximum number of cycles (>= 1)                      */
    double tol;        /* relative residual target (> 0)                       */
    int precision;     /* GNK_PREC_FP64, _DF32, _FMM, _MIXED, _MIXED_DF or
                          _MIXED_FMM                                           */
    int max_refine;    /* MIXED: maximum refinement steps                      */
    double inner_tol;  /* MIXED: relative tolerance of each inner solve        */
    int tile_chunks;   /* tile override of the direct pair-sum kernels (FP64,
                          FP32, double-float): each target tile's sum over the
                          N sources is split into this many chunks of whole
                          source tiles, 1..64 (at most one per tile); 0 = the
                          handle's plan, chosen at build from the SM count.
                          The FMM ignores it.                                */
    int tile_variant;  /* tile override of the batched pair kernels: 1..7
                          selects the (targets per thread, right-hand sides
                          per group) shape in the order of gnk_batch_tuning;
                          0 = the tuned (or default) shape                  */
    int timing;        /* nonzero: gnk_result receives the phase times
                          (CUDA events on `stream`; the call then waits for
                          its last event)                                     */
} gnk_options;

typedef struct gnk_result {
    int status;        /* GNK_OK, GNK_ENOTCONV, GNK_ENONFINITE                  */
    int iterations;    /* Arnoldi steps over all cycles and refinement steps   */
    int cycles;        /* GMRES cycles (restarts + 1) over all inner solves    */
    int refinements;   /* MIXED: refinement steps taken                        */
    int matvecs_fp64;  /* products with the FP64-class (FP64 or DF32) operator */
    int matvecs_fp32;  /* products with the FP32 operator                      */
    double relres;     /* final true relative residual, evaluated in FP64      */
    /* Device time of each phase in ms, with gnk_options.timing set (else 0):
     * setup = deferred precompute (Eone, diagonals) and, for the FMM
     * precisions, the quadtree; rhs = the right-hand side -y (gnk_fbie: with
     * f_B(gamma) from the same sum); solve = GMRES with any refinement;
     * h = h and h_k (gnk_fbie only).  gnk_batch_fbie reports the whole call
     * as solve. */
    double setup_ms;
    double rhs_ms;
    double solve_ms;
    double h_ms;
} gnk_result;

/* Fills `opt` with restart 20, maxit 50, tol 1e-12, FP64, max_refine 10,
 * inner_tol 1e-5, no tile overrides, timing off. */
void gnk_default_options(gnk_options* opt);

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to len-1 characters) and returns its length. */
int gnk_last_error(char* buf, size_t len);

/* Library version string (static storage). */
const char* gnk_version(void);

/* Number of CUDA kernel launches the library has issued in this process
 * (all handles, all devices): a host-side counter for instrumentation. */
unsigned long long gnk_kernel_launches(void);

/* Per-launch device timing for instrumentation.  gnk_profile_enable(1) clears
 * the records and starts recording a CUDA event pair on the launching stream
 * around every kernel launch of the library; gnk_profile_enable(0) stops.
 * gnk_profile_query sums, over the recorded launches of one kind, the number
 * of launches, their device time in ms and their algorithmic work (it waits
 * for the recorded events).  Kinds: 0 FP64, 1 FP32 and 6 double-float
 * pair-sum kernels (work = pair evaluations R N (N-1)), 2 reduction/epilogue,
 * 3 circulant, 4 GMRES vector kernels (work = bytes moved), 5 other, and
 * the FMM kernels: 7 M2L (work = the number of Cauchy sums R, one M2L
 * launch per FMM product), 8 near field (work = near-field pairs evaluated),
 * 9 L2P, 10 the upward pass (P2M and M2M), 11 L2L.  Launches that
 * a converged GMRES cycle turned into no-ops are not counted. */
int gnk_profile_enable(int on);
/* Restricts the recording to the kinds whose bit is set in mask (bit k for
 * kind k; all kinds by default), so that instrumenting the few launches of
 * interest does not add event records to every small launch. */
int gnk_profile_mask(unsigned mask);
int gnk_profile_query(int kind, long long* launches, double* total_ms,
                      double* work);
/* As gnk_profile_query, plus the launches' algorithmic instruction count on
 * their limiting pipe (pair kernels: per pair, FP64 9 + 4R, FP32 6 + 4R,
 * double-float 49 + 48R, R the right-hand sides of the launch; the FMM
 * kernels: FP32-pipe instructions of their double-float arithmetic). */
int gnk_profile_query_ex(int kind, long long* launches, double* total_ms,
                         double* work, double* instr);
/* As gnk_profile_query_ex, plus the algorithmic bytes the launches read and
 * wrote where the kernel is bound by memory rather than by a pipe (the FMM
 * near field from its operator cache: 8 bytes per pair and part of z read);
 * 0 for the other kernels. */
int gnk_profile_query_bytes(int kind, long long* launches, double* total_ms,
                            double* work, double* instr, double* bytes);

/* ---------------------------------------------------------------------------
 * Boundary handle (Sec. 2.1, 2.4; Eqs. eta, A, ti-skp)
 *
 * Builds the device-resident discretised boundary: m1 = m+1 components of n
 * nodes each (n even, n >= 4), N = m1*n.  et, etp, A are eta(t), eta'(t) and
 * A(t) at the nodes; etpp (eta'') and Ap (A') are needed only for the adjoint
 * equation (Eq. bve) and may be NULL otherwise.  bounded = 1 for bounded G
 * (c = +1 in Eq. c), 0 for unbounded G (c = -1).
 * The call also precomputes q = eta'/A, Eone = E q and the diagonals
 * diag(B1) = -(2/n) Im(A Eone), diag(D1) = -(2/n) Re(A Eone) (Sec. 3.3-3.4,
 * listing of FBIE), and, when etpp is given,
 * e = 1 - c - (2/n) Im(E eta') + (2/n) Im(eta''/eta' - A'/A) (Eq. bve), with
 * the corner limit Im(eta''/eta' - A'/A) := 0 where eta' = 0 (graded mesh).
 * A must not vanish; eta' may vanish only at graded-mesh corner nodes.
 * Non-finite input returns GNK_ENONFINITE.  *out receives the handle, which
 * owns all its device memory until gnk_free_boundary.
 * ------------------------------------------------------------------------- */
int gnk_build_boundary(gnk_boundary** out, int m1, int n,
                       const double* et, const double* etp, const double* etpp,
                       const double* A, const double* Ap, int bounded,
                       void* stream);

/* As gnk_build_boundary, with the arithmetic of the precomputed Cauchy sums
 * (Eone and E eta') chosen by `precision` (GNK_PREC_FP64 or GNK_PREC_DF32);
 * gnk_build_boundary uses GNK_PREC_FP64.  With GNK_BUILD_DEFER or-ed into
 * `precision`, those sums are formed by the first call that needs them, and
 * gnk_fbie on a handle without eta'' forms Eone together with E(q gamma) in a
 * single two-right-hand-side launch. */
#define GNK_BUILD_DEFER 0x100
/* With GNK_BUILD_PLAIN or-ed into `precision`, the handle holds the Nystrom
 * discretisation WITHOUT singularity subtraction (the comparison of Sec. 7,
 * Ex. 2): the trapezoidal rule keeps the kernels' diagonal values N(t,t) and
 * M_1(t,t) (Eqs. N-tt, M1-tt), and every operator and solver of the handle uses
 *   I - N      ->  I - B - diag((2 pi/n) N(t,t)),
 *   M          ->  D + L-hat + diag((2 pi/n) M_1(t,t)),
 *   I + N* + J ->  I + diag((2 pi/n) N(t,t)) + B^T + P-hat
 * in place of Eqs. sys, y and sys*.  Needs etpp (Ap NULL means A' = 0); no
 * precomputed Cauchy sum is formed.  At a graded-mesh corner (eta' = 0) both
 * parts of eta''/eta' are taken as 0.  gnk_fbie_backward rejects such a handle
 * (GNK_EINVAL): its geometry derivative is that of the subtracted form. */
#define GNK_BUILD_PLAIN 0x200
int gnk_build_boundary_ex(gnk_boundary** out, int m1, int n,
                          const double* et, const double* etp, const double* etpp,
                          const double* A, const double* Ap, int bounded,
                          int precision, void* stream);

/* Releases the handle and its device memory (NULL is accepted). */
int gnk_free_boundary(gnk_boundary* b);

/* Reports m1 and n of a handle. */
int gnk_boundary_size(const gnk_boundary* b, int* m1, int* n);

/* ---------------------------------------------------------------------------
 * Cauchy sum (Sec. 2.5, Eqs. fmm-1, fmm-E, E-fmm): z = E w,
 *   z_i = sum_{j != i} w_j / (eta_i - eta_j),   i = 1..N,
 * w and z complex (2N doubles).  precision: GNK_PREC_FP64, _FP32, _DF32 or
 * _FMM.
 * ------------------------------------------------------------------------- */
int gnk_cauchy_sum(const gnk_boundary* b, const double* w, double* z,
                   int precision, void* stream);

/* y = (2I + diag(B1) - B) x, the discrete I - N (Eqs. sys, (I-B)x, f_B):
 *   y = 2x - (2/n) Im(A Eone) x + (2/n) Im(A E(q x)).
 * x, y real (N doubles).  precision: GNK_PREC_FP64, _FP32, _DF32 or _FMM. */
int gnk_apply_IminusN(const gnk_boundary* b, const double* x, double* y,
                      int precision, void* stream);

/* y = (D - diag(D1) + Lhat) x, the discrete M (Eqs. y, hD-bt, L-bs):
 *   y = -(2/n) Re(A E(q x)) + (2/n) Re(A Eone) x + Lhat x,
 * Lhat x computed per component by FFT with the exact multipliers of the
 * circulant L (i 2k/n for k < n/2, 0 at k = n/2, i 2(k-n)/n above).
 * x, y real.  precision applies to the pair sum. */
int gnk_apply_M(const gnk_boundary* b, const double* x, double* y,
                int precision, void* stream);

/* y = Lhat x, the block-circulant part alone (Eq. L-bs).  x, y real. */
int gnk_apply_circulant(const gnk_boundary* b, const double* x, double* y,
                        void* stream);

/* y = (diag(e) + B^T + Phat) x, the discrete I + N* + J (Eqs. sys*, BTx, g_B):
 *   y = e x + (2/n) Im(q E(A x)) + Phat x,  Phat x = per-component mean.
 * Needs a handle built with etpp (else GNK_EINVAL). */
int gnk_apply_adjoint(const gnk_boundary* b, const double* x, double* y,
                      int precision, void* stream);

/* ---------------------------------------------------------------------------
 * Solve (I - N) mu = -M gamma (Eq. ie) in the form (2I + diag(B1) - B) mu = -y
 * (Eq. sys) by restarted GMRES (Eq. ie-gmres), device resident (Arnoldi with
 * classical Gram-Schmidt and re-orthogonalisation, Givens rotations, and the
 * convergence test all on the GPU).  gam, mu real (N doubles).  `opt` NULL
 * means gnk_default_options.  `info` (nullable) receives the counters.
 * Returns GNK_OK, or GNK_ENOTCONV with the best iterate written to mu.
 * ------------------------------------------------------------------------- */
int gnk_solve_ie(const gnk_boundary* b, const double* gam, double* mu,
                 const gnk_options* opt, gnk_result* info, void* stream);

/* h = ([D - diag(D1) + Lhat] mu - [2I + diag(B1) - B] gamma) / 2 (Eq. bh),
 * the node values of the piecewise constant h, in FP64.  h (N doubles)
 * receives the node values; hk (m1 doubles, nullable) the mean of h over
 * each component. */
int gnk_compute_h(const gnk_boundary* b, const double* mu, const double* gam,
                  double* h, double* hk, void* stream);

/* The whole computation of the paper's FBIE function (Sec. 3, listing of
 * FBIE): mu solving (I - N) mu = -M gamma and h of Eq. (bh), with the fewest
 * Cauchy sums: E(q gamma) gives both the right-hand side -y and
 * f_B(gamma) = (2I + diag(B1) - B) gamma, and the last true residual of the
 * solve gives f_C(mu) = (D - diag(D1) + Lhat) mu, so h = (f_C(mu) - f_B(gamma))/2
 * needs no further sum.  Products outside the inner GMRES use FP64 for
 * GNK_PREC_FP64 / _MIXED and double-float for _DF32 / _MIXED_DF.  mu, h
 * (N doubles) and hk (m1 doubles, nullable) are outputs.  Returns as
 * gnk_solve_ie. */
int gnk_fbie(const gnk_boundary* b, const double* gam, double* mu, double* h,
             double* hk, const gnk_options* opt, gnk_result* info, void* stream);

/* Solve (I + N* + J) mu = gamma (Eq. ie*) in the form
 * (diag(e) + B^T + Phat) mu = gamma (Eq. sys*) by restarted GMRES
 * (Eq. ie*-gmres).  Needs a handle built with etpp.  Arguments as
 * gnk_solve_ie. */
int gnk_solve_adjoint_ie(const gnk_boundary* b, const double* gam, double* mu,
                         const gnk_options* opt, gnk_result* info,
                         void* stream);

/* ---------------------------------------------------------------------------
 * Differentiation of the FBIE computation (no counterpart in the paper; it
 * uses the transposed system of Eq. sys with the products of Eq. BTx).
 * ------------------------------------------------------------------------- */

/* Solve (2I + diag(B1) - B)^T x = rhs by GMRES, where
 * (2I + diag(B1) - B)^T x = 2x + diag(B1) x - (2/n) Im(q E(A x)).  Arguments
 * as gnk_solve_ie (rhs and x real, N doubles). */
int gnk_solve_ie_transpose(const gnk_boundary* b, const double* rhs, double* x,
                           const gnk_options* opt, gnk_result* info,
                           void* stream);

/* Gradient of a loss L(mu, h, h_k) of the FBIE outputs with respect to the
 * inputs.  Given mu (the solution for gam), gam, grad_mu = dL/dmu and
 * grad_h = dL/dh (N doubles each) and grad_hk = dL/dh_k (m1 doubles, one per
 * component mean h_k; NULL when the loss does not use h_k), writes dL/d eta,
 * dL/d eta', dL/dA (interleaved complex, 2N doubles each: real part =
 * derivative with respect to the real part of the input, imaginary part =
 * derivative with respect to its imaginary part) and dL/dgam (N doubles).
 * Method: grad_h + grad_hk[k]/n on the nodes of component k (h_k is a mean),
 * one transposed solve lambda = K^-T (grad_mu + M^T grad_h / 2) with
 * K = 2I + diag(B1) - B and M = D - diag(D1) + Lhat, then one FP64 pass of six
 * Cauchy sums and six sums of the derivative kernel 1/(eta_i - eta_j)^2.
 * `opt` controls the transposed solve (its precision also sets the arithmetic
 * of M^T).  Host arrays are staged through temporary device buffers.  Returns
 * GNK_OK or GNK_ENOTCONV (gradient from the best iterate). */
int gnk_fbie_backward(const gnk_boundary* b, const double* mu, const double* gam,
                      const double* grad_mu, const double* grad_h, const double* grad_hk,
                      double* grad_et, double* grad_etp, double* grad_A,
                      double* grad_gam, const gnk_options* opt,
                      gnk_result* info, void* stream);

/* ---------------------------------------------------------------------------
 * Cauchy integral formula with singularity subtraction (Sec. 5, Eqs. cauchy4
 * and cauchy6): values at points z of G of the function f analytic in G whose
 * boundary values f(eta_j) are given, from the trapezoidal sums
 *   S1(z) = sum_j f_j eta'_j / (z - eta_j),   S2(z) = sum_j eta'_j / (z - eta_j)
 * over all N nodes of the handle:
 *   bounded G:   f(z) = S1 / S2,
 *   unbounded G: f(z) = (f_inf - S1 / (n i)) / (1 - S2 / (n i)).
 * z (nz points) and fz are interleaved complex arrays of 2 nz doubles, f of
 * 2N doubles; host or device pointers (host arrays are copied through a
 * temporary device buffer).  finf (2 doubles: f at infinity) is read on the
 * host and used only for unbounded G; NULL means 0.  precision: GNK_PREC_FP64
 * or GNK_PREC_DF32.  Points on the boundary itself are not excluded: a point
 * equal to a node returns a non-finite value there.  nz == 0 returns GNK_OK
 * without a launch and reads no array; nz < 0, NULL arrays (nz > 0) or
 * another precision return GNK_EINVAL.  Allocates a temporary workspace of 2 nz x (<= 32 chunks)
 * complex partial sums and synchronises `stream` before returning.
 * ------------------------------------------------------------------------- */
int gnk_cauchy_eval(const gnk_boundary* b, int nz, const double* z,
                    const double* f, const double* finf, double* fz,
                    int precision, void* stream);

/* ---------------------------------------------------------------------------
 * Conformal maps onto slit domains by the FBIE route of Sec. 7, Ex. 3 (bounded
 * G) and Ex. 4 (unbounded G), the method of the paper's references for those
 * examples: for a point alpha of G and theta_k = pi/2 (circular slit) or 0
 * (radial slit) per boundary (theta_0 = pi/2 for the outer boundary of a
 * bounded G),
 *   gamma = -Re[e^{i(pi/2 - theta)} log(eta - alpha)]   (arg continuous along
 *           each boundary),
 *   bounded G:   A = e^{i(pi/2 - theta)} (eta - alpha),
 *   unbounded G: A = e^{i(pi/2 - theta)}                  (Eq. A),
 * then (mu, h, h_k) of gnk_fbie on a handle built with this A give the analytic
 * f with A f = gamma + h + i mu (f(inf) = 0 for unbounded G) and the map
 *   bounded G:   w(z) = e^{-h_0} (z - alpha) exp((z - alpha) f(z)),
 *                onto the unit disk: |w| = 1 on the outer boundary, w(alpha) = 0,
 *                w'(alpha) = e^{-h_0} > 0, a circular-slit boundary maps to
 *                |w| = e^{h_k - h_0};
 *   unbounded G: w(z) = (z - alpha) exp(f(z)),
 *                onto the plane with slits: w(alpha) = 0, w(z) = z + O(1) at
 *                infinity, a circular-slit boundary maps to |w| = e^{h_k};
 * a radial-slit boundary maps to arg w = const.
 *
 * gnk_slit_map_data: A (2N doubles) and gamma (N) from eta (2N), alpha (2
 *   doubles, read on the host), theta (m1 doubles, one per boundary) and
 *   bounded (1: bounded G, 0: unbounded G).
 * gnk_slit_map: w at the nodes (2N doubles) from gamma, mu, h (N each) and h_k
 *   (m1) of the solve; the handle must be built with that A (its boundedness
 *   selects the formula).
 * gnk_slit_map_eval: w at nz points z of G (2 nz doubles in, 2 nz out), f from
 *   the Cauchy formula (gnk_cauchy_eval's sums with f(inf) = 0, precision
 *   GNK_PREC_FP64 or GNK_PREC_DF32).
 * Arrays may be host or device pointers (host arrays are staged); the calls
 * synchronise `stream`.  GNK_EINVAL for NULL arrays, nz < 0 or m1, n out of
 * range.
 * ------------------------------------------------------------------------- */
int gnk_slit_map_data(int m1, int n, const double* et, const double* alpha,
                      const double* theta, int bounded, double* A, double* gam,
                      void* stream);
int gnk_slit_map(const gnk_boundary* b, const double* alpha, const double* gam,
                 const double* mu, const double* h, const double* hk, double* w,
                 void* stream);
int gnk_slit_map_eval(const gnk_boundary* b, const double* alpha,
                      const double* gam, const double* mu, const double* h,
                      const double* hk, int nz, const double* z, double* wz,
                      int precision, void* stream);

/* ---------------------------------------------------------------------------
 * The same slit maps by solves of the adjoint equation only (Sec. 7, Ex. 3 and
 * Ex. 4: the comparison route of the FBIEad function, whose map formulas the
 * paper leaves to its references; the steps below follow from the identities
 * of the generalized Neumann kernel formed with A~ = eta'/A (Eqs. A*, Nt-N*)
 * and Cauchy's theorem).  theta_k = pi/2 (circular slit) or 0 (radial slit),
 * pi/2 on the outer boundary of a bounded G.  With w = (z - alpha) exp(omega):
 *   psi, the derivative of the boundary correspondence (th' where
 *     w = R_k e^{i th_k(t)} on a circular boundary, -(log rho_k)' where
 *     w = rho_k(t) e^{i phi_k} on a radial one), solves Eq. (ie*)
 *     (I + N* + J) psi = e_0 for bounded G and
 *     (I + N* + J) psi = 2 Im[A~/(eta - alpha)] for unbounded G;
 *   S, its antiderivative along each boundary with S = 0 at t = 0, from the
 *     FFT of its trigonometric interpolant (a direct circulant product when n
 *     is not a power of two up to 4096);
 *   psi_j solves (I + N* + J) psi_j = e_j (e_j = 1 on boundary j, 0 elsewhere),
 *     j = 0..m, and T_j = (1/n) sum_i c_i om_i psi_j,i with c = i (circular)
 *     or -1 (radial) and om = omega without its per-boundary constants
 *     (circular: -log|eta - alpha| + i (S - arg(eta - alpha)); radial:
 *     -S - log|eta - alpha| - i arg(eta - alpha), arg continuous along each
 *     boundary); rho = log w'(alpha) = Im T_0 for bounded G, 0 for unbounded G;
 *   circular k: R_k = e^{rho - Im T_k}, th_k(0) = Re T_k,
 *               w = R_k e^{i (th_k(0) + S)};
 *   radial k:   phi_k = Im T_k, w = e^{rho + Re T_k - S} e^{i phi_k}.
 * Bounded G: m + 1 solves (psi = psi_0); unbounded G: m + 2.  The map is the
 * one of gnk_slit_map: onto the unit disk with w(alpha) = 0, w'(alpha) > 0
 * (bounded G) or onto the plane with w = z + O(1) at infinity (unbounded G).
 *
 * gnk_slit_map_adjoint_data: A' (2N doubles) = e^{i(pi/2 - theta)} eta' for
 *   bounded G, 0 for unbounded G, from eta' (2N) and theta (m1): with
 *   gnk_slit_map_data's A and eta'' the handle for this route is built by
 *   gnk_build_boundary(_ex).
 * gnk_slit_map_adjoint: on such a handle, for alpha (2 doubles, read on the
 *   host) and theta (m1 doubles, host or device, read on the host), writes w at
 *   the nodes (2N doubles); optionally (each nullable) omega at the nodes (2N),
 *   psi (N) and params (m1 + 1: R_k on a circular boundary, phi_k on a radial
 *   one, then w'(alpha) for bounded G or 1).  `opt` controls every GMRES solve
 *   (any precision of gnk_solve_adjoint_ie); `info` sums the solves' counts
 *   and keeps the largest final residual.  Returns GNK_OK, GNK_ENOTCONV (a
 *   solve stopped at maxit; the outputs are written), GNK_ENONFINITE,
 *   GNK_EINVAL (NULL handle or arrays, a handle without eta'', theta not pi/2
 *   or 0, theta_0 != pi/2 for bounded G, bad options) or GNK_ENOMEM.
 *   Allocates a workspace of about 6N + 2 m1 + n doubles from the pool.
 * gnk_slit_map_adjoint_eval: w at nz points z of G (2 nz doubles in and out)
 *   from omega at the nodes: omega(z) by the Cauchy formula (gnk_cauchy_eval,
 *   omega(inf) = 0 for unbounded G; precision GNK_PREC_FP64 or GNK_PREC_DF32),
 *   then w = (z - alpha) exp(omega(z)).
 * Host arrays are staged; the calls synchronise `stream`.
 * ------------------------------------------------------------------------- */
int gnk_slit_map_adjoint_data(int m1, int n, const double* etp,
                              const double* theta, int bounded, double* Ap,
                              void* stream);
int gnk_slit_map_adjoint(const gnk_boundary* b, const double* alpha,
                         const double* theta, const gnk_options* opt,
                         double* w, double* omega, double* psi,
                         double* params, gnk_result* info, void* stream);
int gnk_slit_map_adjoint_eval(const gnk_boundary* b, const double* alpha,
                              const double* omega, int nz, const double* z,
                              double* wz, int precision, void* stream);

/* ---------------------------------------------------------------------------
 * Batched FBIE over many independent domains and right-hand sides (no
 * counterpart in the paper: many instances of Sec. 3 solved together).
 *
 * Domain d has m1[d] components of n[d] nodes (N_d = m1[d] n[d]), nrhs[d]
 * right-hand sides and boundedness bounded[d]; et, etp, A hold the domains'
 * nodes one after the other (interleaved complex, 2 sum_d N_d doubles).
 * System s = (d, r) is the r-th right-hand side of domain d; batch vectors
 * (gamma, mu, h) store the systems one after the other, domain by domain and
 * right-hand side by right-hand side (length L = sum_d nrhs[d] N_d), and hk
 * stores the m1[d] component means of each system in the same order.
 * Each operator product is one persistent kernel launch over a work list of
 * (domain, target tile, right-hand-side group) items; the Arnoldi steps of a
 * restart cycle are captured in a CUDA graph.  With autotune != 0 the tile
 * shapes (targets per thread, right-hand sides per group) of the FP32 and
 * double-float kernels are chosen by timing each variant on a sample of the
 * batch; otherwise fixed defaults are used.  Arrays may be host or device
 * memory.
 * ------------------------------------------------------------------------- */
typedef struct gnk_batch gnk_batch;

int gnk_build_batch(gnk_batch** out, int ndomains, const int* m1, const int* n,
                    const int* nrhs, const int* bounded, const double* et,
                    const double* etp, const double* A, int autotune,
                    void* stream);
int gnk_free_batch(gnk_batch* b);

/* Vector length L, number of systems, and length of the hk array. */
int gnk_batch_sizes(const gnk_batch* b, long long* vec_len, int* systems,
                    int* hk_len);

/* Chosen tile shapes and the tuning times (ms) of the seven variants:
 * FP32 (T, RG) = (1,8), (2,4), (2,8), (4,4), double-float (1,2), (1,4), (2,2). */
int gnk_batch_tuning(const gnk_batch* b, int* fp32_targets, int* fp32_group,
                     int* df_targets, int* df_group, float* variant_ms);

/* y = (2I + diag(B1) - B) x for every system of the batch (Eq. sys), with FP32
 * (GNK_PREC_FP32) or double-float (GNK_PREC_DF32) pair sums; x and y are batch
 * vectors (host or device).  One persistent launch. */
int gnk_batch_apply_IminusN(const gnk_batch* b, const double* x, double* y,
                            int precision, void* stream);

/* mu and h of every system (FBIE: Eqs. sys, y, bh).  opt->precision
 * GNK_PREC_MIXED_DF (the default when opt is NULL): FP32 pair sums inside
 * GMRES and double-float refinement, every product one persistent launch over
 * the whole batch.  GNK_PREC_FMM: each domain solved by the single-domain FBIE
 * path with FMM products (Sec. 2.5; domains of fewer than 4096 nodes with
 * double-float direct sums), one quadtree and its caches per domain kept with
 * the batch, the domains taken largest first by 8 host worker threads with a
 * CUDA stream each, so that several domains' products share the GPU.  Each
 * system stops when its own ||b - A mu|| <= tol ||b||.  info->relres is the
 * largest final relative residual; relres_per_system (nullable, one double
 * per system) receives each.  hk is nullable. */
int gnk_batch_fbie(const gnk_batch* b, const double* gam, double* mu,
                   double* h, double* hk, const gnk_options* opt,
                   gnk_result* info, double* relres_per_system, void* stream);

/* ---------------------------------------------------------------------------
 * Cauchy sum without any device allocation (no counterpart in the paper).
 *
 * z = E w exactly as gnk_cauchy_sum computes it in FP64, for callers that
 * cannot allocate device memory: plugins running inside a host application
 * that owns all device memory and forbids allocations of its own, and
 * real-time loops where an allocation's implicit device synchronisation, or
 * its possible failure, is not acceptable.  No handle is needed: et (eta at
 * the N nodes), w and z are interleaved complex arrays of 2N doubles that
 * must already be in device memory of the current device (host pointers and
 * memory of another GPU return GNK_EINVAL; nothing is staged or copied).  The
 * split-source partial sums go to a fixed 4 MiB array inside the library's
 * device image, which every GPU that loads the library keeps until the
 * process exits; it limits N to 1..65536 (larger N returns GNK_EINVAL before
 * any launch).  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress), so make the first call on each device
 * before any stream capture.  All calls share the array: calls whose kernels
 * can overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Each call overwrites every entry it reads, so no
 * clearing is needed between calls.  Never calls cudaMalloc or cudaFree.
 * The library cannot check the arrays' lengths: each must hold at least N
 * complex values.
 * ------------------------------------------------------------------------- */
int gnk_cauchy_sum_noalloc(int N, const double* et, const double* w,
                           double* z, void* stream);

/* ---------------------------------------------------------------------------
 * Diagnostics for tests (no counterpart in the paper).
 *
 * gnk_debug_recip_f64: y_lib[i] = the FP64 reciprocal that the pair-sum
 *   kernels use for 1/|d|^2 (the hardware seed refined by the series
 *   y0 (1 + e + e^2), e = 1 - x y0) and y_div[i] = 1.0 / x[i] by CUDA's IEEE
 *   division, for n doubles x (device arrays, n >= 0; GNK_EINVAL for host
 *   pointers).  Asynchronous on `stream`.
 * gnk_debug_split_f64: hi[i], lo[i] = the double-float split of x[i] that the
 *   FMM's gather and evaluation kernels use (from the bits of x: hi = x
 *   truncated to 24 significant bits, lo = the next 23 bits, so
 *   |x - (hi + lo)| < 2^-46 |x| for 2^-80 <= |x| < 2^101; other values take
 *   hi = (float)x, lo = (float)(x - hi)), for n doubles x (device arrays,
 *   n >= 0; GNK_EINVAL for host pointers).  Asynchronous on `stream`.
 * gnk_debug_barrier_fault: test hook of the bounded grid-barrier waits inside
 *   the cooperative Arnoldi step of every later GMRES solve (Sec. 3.5).  With
 *   skip_block >= 0 that block passes each barrier without arriving, so the
 *   other blocks' waits run out after spin_limit polls (0 = the default
 *   limit, 2^20), they set an error flag and return, and the solve returns
 *   GNK_ECUDA with the message "a grid barrier of the Arnoldi step timed
 *   out"; no kernel faults and the device stays usable.  (-1, 0) restores
 *   normal operation.  Process-wide; not for use while solves run on other
 *   threads.  GNK_EINVAL for skip_block < -1 or spin_limit < 0.
 * ------------------------------------------------------------------------- */
int gnk_debug_recip_f64(int n, const double* x, double* y_lib, double* y_div, void* stream);
int gnk_debug_split_f64(int n, const double* x, float* hi, float* lo, void* stream);
int gnk_debug_barrier_fault(int skip_block, int spin_limit);

#ifdef __cplusplus
}
#endif

#endif /* GNK_H */

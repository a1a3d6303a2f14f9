/*
 * mqct.h -- C ABI of the GB300 MQCT trajectory library.
 *
 * The library propagates many mixed quantum/classical (Ehrenfest mean-field)
 * trajectories of an atom + rigid rotor collision on one GPU and turns their
 * final state populations into state-to-state cross sections, following
 * Joy, Mandal, Bostan, Dubernet & Babikov, arXiv 2312.02322:
 *
 *   Eq. 4     a_n(t): amplitudes in the interaction picture, c_n = exp(-i E_n t) a_n
 *   Eq. 5     da/dt = -i exp(iEt) M(R) c  +  (dPhi/dt / 2) (J+ - J-) a      (Coriolis, m +- 1)
 *   Eq. 6     M(R): real, symmetric, block-diagonal in m
 *   Eqs. 7-10 dR/dt = P_R/mu, dPhi/dt = P_Phi/(mu R^2),
 *             dP_R/dt = -Re(c^dag M'(R) c) + P_Phi^2/(mu R^3),
 *             dP_Phi/dt = Re(c^dag (J+ - J-) M(R) c)
 *   Eq. 12    M(R) = sum_lambda v_lambda(R) G^lambda   (angular expansion of the PES)
 *   Sec. III  v_lambda(R) (and thus M(R)) interpolated by cubic splines on an R grid
 *   Sec. II   cross sections: final |a|^2 summed over the final level, averaged over the
 *             initial degenerate states and integrated over impact parameter
 *
 * Conventions shared by every call:
 *   - atomic units throughout: hartree, bohr, electron masses, atomic units of time;
 *   - arrays are C-contiguous, row-major; "[A][B]" means A slow, B fast;
 *   - a pointer argument may be a host or a device pointer unless stated otherwise
 *     (the library asks the CUDA driver which one it is);
 *   - the caller keeps ownership of every array it passes; nothing is retained after
 *     the call returns except what mqct_create_system copies into the system;
 *   - no call aborts the process or traps the GPU: failures are reported by the
 *     returned status and a thread-local message (mqct_last_error);
 *   - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 *
 * Readings of the paper where its printed text is garbled or silent:
 *   - Coriolis term of Eq. 5: the anti-Hermitian form above, i.e. the quantum
 *     Hamiltonian H_rot + V - dPhi/dt J_y, J_y = (J+ - J-)/(2i);
 *   - torque of Eq. 10: i<[J_y, V]> = Re(c^dag (J+ - J-) M c), the form for which the
 *     total energy and P_Phi + <J_y> are conserved;
 *   - initial state: a = e_{init_state}, R = r0, Phi = 0, P_Phi = b sqrt(2 mu E),
 *     P_R = -sqrt(2 mu (E - M_ss(r0)) - P_Phi^2 / r0^2);
 *   - splines: clamped cubic on a uniform grid; interval k = floor((R - r_min)/h) clamped
 *     to [0, n_grid-2]; outside the grid the end cubic is extrapolated;
 *   - integrator: classical 4-stage RK4 with fixed dt, stage times t, t+dt/2, t+dt/2, t+dt,
 *     t = n dt; a trajectory ends after the first step that ends with R >= r_end and
 *     P_R > 0, or after max_steps steps.
 */
#ifndef MQCT_H
#define MQCT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mqct_system_s *mqct_system; /* opaque; owns all of its device memory */

typedef enum {
    MQCT_OK = 0,
    MQCT_ERR_INVALID_ARG = 1, /* a size, pointer or value failed validation           */
    MQCT_ERR_OOM = 2,         /* host or device allocation failed                      */
    MQCT_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    MQCT_ERR_UNSUPPORTED = 4, /* combination of options not implemented                */
    MQCT_ERR_TIMEOUT = 5,     /* a bounded device wait ran out                          */
    MQCT_ERR_TRAJ = 6         /* the call ran, but at least one trajectory status != 0 */
} mqct_status;

/* Coupling evaluation (both are the same mathematics, Eq. 12 and Sec. III):
 *   PLAIN:      spline table of every structurally non-zero M_nm(R) (M is block-diagonal
 *               in m, Eq. 6), evaluated per trajectory and fused with the mat-vec;
 *   FACTORISED: M(R) c = sum_lambda v_lambda(R) (G^lambda c), G^lambda constant. */
typedef enum { MQCT_PATH_PLAIN = 0, MQCT_PATH_FACTORISED = 1 } mqct_path;

/* Precision of the amplitudes and of the coupling contraction.  Phase arguments E_n t,
 * the classical variables and the conserved-quantity bookkeeping are FP64 in every mode.
 * MQCT_FP32 on the FACTORISED path runs the persistent batched kernel (amplitudes of a few
 * trajectories in each CTA's shared memory, bases up to ~3000 states); MQCT_FP32 on the PLAIN path
 * runs the stage-synchronous sparse path for bases of any size (amplitudes of every trajectory in
 * flight in device memory, an FP32 spline table of every retained M_nm evaluated per element and
 * trajectory, the logarithmic grid and the truncation of Sec. III available).  MQCT_BF16X3 (FACTORISED
 * only) runs the stage-synchronous tensor-core path.  Both stage-synchronous paths run every
 * trajectory under one CUDA graph with a conditional loop; with the environment variable
 * MQCT_TC_HOST_LOOP=1 the same kernels are launched from a host loop instead (for profilers that do
 * not follow conditional graph nodes; same arithmetic). */
typedef enum { MQCT_FP64 = 0, MQCT_FP32 = 1, MQCT_BF16X3 = 2 } mqct_precision;

/* per-trajectory status bits (mqct_diag.status) */
#define MQCT_TRAJ_MAX_STEPS 1   /* max_steps reached before the stop rule (e.g. orbiting)   */
#define MQCT_TRAJ_TABLE_RANGE 2 /* some stage had R < r_min (end cubic extrapolated)        */
#define MQCT_TRAJ_NONFINITE 4   /* a non-finite value appeared; the trajectory was stopped  */
#define MQCT_TRAJ_TIMEOUT 8     /* a bounded device wait ran out while running it           */
#define MQCT_TRAJ_INVALID 16    /* device-resident trajectory failed validation; not run    */
#define MQCT_TRAJ_CKPT 32       /* adjoint: the forward pass outran its checkpoint storage  */

/* mqct_system_desc.flags */
#define MQCT_PRESCRIBED_TRAJ 1  /* prescribed classical trajectory (FP64 systems only): instead of
   the Ehrenfest motion of Eqs. 7-10, each trajectory follows the straight line
   R(t) = sqrt(b^2 + v^2 (t - t_0)^2), dPhi/dt = b v / R^2, with v = sqrt(2 e_coll / mu) and
   t_0 = max_steps dt / 2 (time-symmetric about the middle of the run), for exactly max_steps RK4
   steps (r0 and r_end are not used; the mean field does not act back on the motion).  The
   quantum equation (Eqs. 4-6) is integrated along it.  This is the setting in which microscopic
   reversibility (Eq. 19) holds exactly for the discrete propagator.  P_R = P_Phi = 0 in the
   diagnostics' energy. */
#define MQCT_DECOUPLED_TRAJ 2   /* decoupled classical motion (FP64 systems only; the AT-MQCT
   decoupling of Sec. III, whose equations the paper does not give, in this reading): R, Phi, P_R,
   P_Phi follow Eqs. 7-10 with the mean field replaced by the isotropic potential alone -- the sum
   v_iso(R) of the expansion terms whose G is the identity, which must exist -- and no torque, so the
   path does not depend on the amplitudes; the amplitudes follow Eqs. 4-6 (Coriolis term included)
   along it.  P_R starts from e_coll - v_iso(r0).  The diagnostics then track the classical energy
   P_R^2/2mu + P_Phi^2/(2 mu R^2) + v_iso(R) and P_Phi, both conserved by this motion. */

/* Description of one atom + rotor system.  All pointers are HOST pointers, read and
 * copied during mqct_create_system only. */
typedef struct {
    int32_t n_states;        /* N >= 1                                                        */
    const double *energy;    /* [N] internal energies E_n (hartree); equal within a level    */
    const int32_t *level;    /* [N] non-degenerate level id in [0, n_levels); sigma is per level */
    const int32_t *j;        /* [N] angular momentum label for the Coriolis ladder;
                                j < 0 switches the Coriolis term off for the state            */
    const int32_t *m;        /* [N] projection m (|m| <= j when j >= 0); M is block-diagonal in m */
    double mu;               /* reduced mass (electron masses), > 0                          */
    int32_t n_terms;         /* L >= 1 expansion terms of Eq. 12                             */
    const double *G;         /* [L][N][N] real symmetric G^lambda, or NULL to use triplets   */
    int64_t g_nnz;           /* triplet form (used when G == NULL): entries (term,row,col,val); */
    const int32_t *g_term;   /*   each stored entry of a symmetric matrix must appear for both */
    const int32_t *g_row;    /*   (row,col) and (col,row); duplicates are summed              */
    const int32_t *g_col;
    const double *g_val;
    int32_t n_grid;          /* >= 4 grid points (grid_kind below)                            */
    double r_min, r_max;
    const double *v;         /* [L][n_grid] v_lambda(R_k) (hartree)                          */
    const double *dv_ends;   /* [L][2] dv_lambda/dR at r_min and r_max (clamped spline)      */
    int32_t n_params;        /* P >= 0 parameters theta for mqct_adjoint                     */
    const double *dv_dparam; /* [P][L][n_grid] d v_lambda(R_k) / d theta_p, or NULL if P = 0 */
    const double *ddv_ends;  /* [P][L][2] their R-derivatives at both ends                   */
    int32_t path;            /* mqct_path                                                    */
    int32_t precision;       /* mqct_precision                                               */
    int32_t flags;           /* 0, MQCT_PRESCRIBED_TRAJ or MQCT_DECOUPLED_TRAJ                */
    int32_t grid_kind;       /* MQCT_GRID_UNIFORM, or MQCT_GRID_LOG (below)                   */
    double trunc_threshold;  /* PLAIN path: M_nm dropped when |M_nm(R)| <= threshold at both  */
    double trunc_r[2];       /*   trunc_r (hartree, bohr; Sec. III); <= 0 keeps every element */
    double adapt_tol;        /* > 0: adaptive step control (FP64 systems; below), 0: fixed dt   */
    int32_t adapt_hmax;      /* largest adaptive step in units of dt: a power of 2 in [1, 1024],
                                0 = 16                                                        */
} mqct_system_desc;

/* Adaptive step control (FP64 systems; the paper's ADAPTOL predictor of Sec. III is not given, this
 * is the reading used): step doubling -- one RK4 step of h against two of h/2 from the same state,
 * error = max_n |a_n(two halves) - a_n(one step)|.  The two-half result is kept when the error is at
 * most adapt_tol or h is already the trajectory's dt (the smallest step); otherwise h is halved and
 * the step retried from the same state.  After an accepted step h doubles, up to adapt_hmax dt, when
 * the error was at most adapt_tol / 64.  h starts at adapt_hmax dt.  max_steps and the diagnostics'
 * steps count accepted steps; t_final is the time reached.  Not with MQCT_PRESCRIBED_TRAJ. */

/* R grids (Sec. III).  MQCT_GRID_UNIFORM: R_k = r_min + k (r_max - r_min)/(n_grid - 1), splines
 * clamped cubics in R.  MQCT_GRID_LOG: R_k = r_min (r_max/r_min)^(k/(n_grid - 1)), r_min > 0 (the
 * paper's logarithmic spacing); the splines are clamped cubics in ln R on its uniform grid (end
 * slopes R dv/dR from dv_ends), R-derivatives by the chain rule.  The logarithmic grid runs on
 * MQCT_FP64 systems (both paths) and on MQCT_FP32 systems of the PLAIN path.
 * Truncation (PLAIN path only): M_nm(R) = sum_lambda v_lambda(R) G^lambda_nm is evaluated from the
 * splines at trunc_r[0] and trunc_r[1]; an element whose magnitude is <= trunc_threshold at both is
 * dropped for the whole propagation (the paper keeps |M| > 1 cm^-1 at 6.03 and 7.11 bohr). */
#define MQCT_GRID_UNIFORM 0
#define MQCT_GRID_LOG 1

/* One trajectory (Sec. III: collision energy, impact parameter, initial state). */
typedef struct {
    double e_coll;      /* collision energy (hartree), > 0                     */
    double b;           /* impact parameter (bohr), >= 0                       */
    double r0;          /* initial R (bohr), > 0                               */
    double r_end;       /* stop once R >= r_end with P_R > 0                   */
    double dt;          /* RK4 step (a.u. of time), > 0                        */
    int32_t init_state; /* index in [0, N) of the system's caller state order  */
    int32_t max_steps;  /* >= 0                                                */
    int32_t system_idx; /* index into the `systems` array of mqct_propagate    */
} mqct_traj;

/* Per-trajectory diagnostics.  Deviations are maxima over the states at the start of
 * every step and the final state: | sum|a|^2 - 1 |, | E_tot - E_tot(0) | with
 * E_tot = P_R^2/(2mu) + P_Phi^2/(2mu R^2) + sum E|a|^2 + Re(c^dag M c), and
 * | (P_Phi + <J_y>) - (P_Phi + <J_y>)(0) |. */
typedef struct {
    int32_t steps;   /* RK4 steps taken                 */
    int32_t status;  /* MQCT_TRAJ_* bits; 0 = OK        */
    double norm_dev;
    double energy_dev;
    double angmom_dev;
    double t_final;  /* steps * dt                       */
} mqct_diag;

/* Read-only facts about a created system (host struct filled by mqct_system_info). */
typedef struct {
    int32_t n_states, n_levels, n_terms, n_grid, n_blocks, max_block;
    int32_t path, precision;
    int64_t table_nnz;        /* PLAIN: structurally non-zero M_nm per interval          */
    int64_t table_bytes;      /* PLAIN: device bytes of the spline table                 */
    int64_t glambda_nnz;      /* FACTORISED: sum over lambda of non-zero G^lambda entries */
    int64_t device_bytes;     /* all device memory the system owns                        */
    int32_t n_coupling_terms; /* FACTORISED: terms stored as matrices (identity terms are not) */
    int32_t n_row_tiles;      /* BF16X3: 128-row tiles of whole m-blocks                   */
    int64_t tc_kchunks;       /* BF16X3: non-zero 16-column K chunks over terms and tiles  */
    int64_t trunc_dropped;    /* PLAIN: elements M_nm dropped by the truncation           */
    int32_t grid_kind;        /* MQCT_GRID_UNIFORM or MQCT_GRID_LOG                        */
    int32_t reserved;
} mqct_system_info_t;

/* Parameters of the built-in atom + linear rotor system (helper for users and tests):
 * E_j = B j (j+1), states (j, m) for j <= jmax in j-major order s = j^2 + j + m,
 * V(R, theta) = sum_l A_l exp(-beta_l R) P_l(cos theta) - C6 R^-6 (1 - exp(-(R/Rd)^6)),
 * G^lambda_{(j''m),(j'm)} = <j'' m|P_lambda|j' m> (Eq. 15).  With with_params != 0 the
 * derivative tables for theta = (A_0..A_{L-1}, beta_0..beta_{L-1}) are filled (P = 2L). */
typedef struct {
    int32_t jmax;        /* 0..500 (N = (jmax+1)^2 <= 251 001) */
    double bconst;       /* hartree            */
    double mu;           /* electron masses    */
    int32_t n_terms;     /* L <= 16            */
    double A[16];        /* hartree            */
    double beta[16];     /* 1/bohr             */
    double c6;           /* hartree bohr^6     */
    double rd;           /* bohr               */
    int32_t n_grid;
    double r_min, r_max;
    int32_t with_params;
    int32_t path, precision;
    int32_t grid_kind;        /* MQCT_GRID_UNIFORM or MQCT_GRID_LOG: tabulation grid of v_lambda */
    double trunc_threshold;   /* copied into the description (PLAIN path truncation)            */
    double trunc_r[2];
} mqct_diatom_params;

/* Build the description of the atom + linear rotor system above.  Allocates the host
 * arrays of *out (released by mqct_free_desc); G is returned in triplet form.
 * Host-only: needs no GPU.  Errors: MQCT_ERR_INVALID_ARG (jmax outside [0, 500], n_terms outside
 * [1, 16], n_grid < 4, r_max <= r_min, mu <= 0), MQCT_ERR_OOM. */
mqct_status mqct_build_diatom(const mqct_diatom_params *p, mqct_system_desc *out);
/* Parameters of the built-in atom + rigid asymmetric top system (helper for users and tests).
 * Rotor states (Eq. 1): psi_{J tau M} = sum_K b_K sqrt((2J+1)/(8 pi^2)) D^{J*}_{MK}, the b_K
 * diagonalising A Ja^2 + B Jb^2 + C Jc^2 (K = projection on the a axis); within one J the
 * 2J+1 levels are labelled tau = -J..J in ascending energy.  The basis keeps whole levels (all
 * 2J+1 values of M) for J <= jmax in ascending energy (ties: smaller J first) while the number
 * of states stays <= max_states; states are level-major, M = -J..J within a level, and each
 * level's eigenvector has its largest component in Wang's symmetrised functions positive.
 * PES: V = sum_t v_t(R) f_t with v_t = coef_t exp(-beta_t R) (plus the damped dispersion
 * -C6 R^-6 (1 - exp(-(R/Rd)^6)) on term 0) and the real angular functions
 *   f_t = (D^{lam*}_{0 mu} + (-1)^mu D^{lam*}_{0,-mu}) / (1 + delta_{mu 0}),  0 <= mu <= lam,
 * i.e. P_lam(cos beta) for mu = 0 and 2 d^lam_{0 mu}(beta) cos(mu gamma) otherwise (the +-mu
 * combination of Eq. 14 for an atom partner).  G^t = <J'' tau'' M | f_t | J' tau' M> (the Eq. 16
 * integrals) is real symmetric and block-diagonal in M.  With with_params != 0 the derivative
 * tables for theta = (coef_0..coef_{L-1}, beta_0..beta_{L-1}) are filled (P = 2L). */
typedef struct {
    int32_t jmax;        /* 0..20                                                  */
    double A, B, C;      /* rotational constants (hartree), A >= B >= C > 0, A > C */
    int32_t max_states;  /* >= 1                                                    */
    double mu;           /* reduced mass (electron masses)                         */
    int32_t n_terms;     /* L in [1, 64]                                           */
    int32_t lam[64];     /* lambda_t in [0, 8]                                     */
    int32_t mproj[64];   /* mu_t in [0, lambda_t]                                  */
    double coef[64];     /* hartree                                                */
    double beta[64];     /* 1/bohr                                                 */
    double c6;           /* hartree bohr^6                                         */
    double rd;           /* bohr                                                   */
    int32_t n_grid;
    double r_min, r_max;
    int32_t with_params;
    int32_t path, precision;
    int32_t *tau_out;    /* optional HOST array of (jmax+1)^2 entries: tau of each kept level */
} mqct_asym_params;

/* Build the description of the atom + asymmetric top system above (host only, no GPU).
 * Allocates the host arrays of *out (released by mqct_free_desc); G in triplet form.
 * Errors: MQCT_ERR_INVALID_ARG (a bound above violated, or max_states below the first
 * level), MQCT_ERR_OOM. */
mqct_status mqct_build_asym_top(const mqct_asym_params *p, mqct_system_desc *out);

/* Parameters of the built-in asymmetric top + linear rotor system (the molecule-molecule coupling of
 * Sec. II; helper for users and tests).  Composite states (Eq. 3)
 *   |n m> = sum_{m1} C^{j m}_{j1 m1 j2 m-m1} psi_{j1 tau1 m1}(Lambda_1) Y^{j2}_{m-m1}(Lambda_2),
 * n = {j, j1, tau1, j2}: molecule 1 levels (j1, tau1) of Eq. 1 for j1 <= j1max (ascending j1, then
 * ascending energy), each combined with every j2 of the list, every total j in |j1 - j2| .. j1 + j2
 * and m = -j..j (in that order); level id = (molecule-1 level) * n_j2 + index of j2, energy
 * E_{j1 tau1} + bconst2 j2 (j2 + 1); the Coriolis ladder acts on the total j.  PES (Eq. 12) with the
 * angular functions tau_{lam1 mu1 lam2 lam} of Eq. 13 and v_t(R) = coef_t exp(-beta_t R) (term 0 adds
 * the damped dispersion -C6 R^-6 (1 - exp(-(R/Rd)^6))); G^t = <n'' m|tau_t|n' m> (Eq. 14 with the
 * integrals of Eqs. 15-16; here evaluated by Gauss-Legendre quadrature over the polar angles). */
typedef struct {
    double A, B, C;          /* molecule 1 rotational constants (hartree), A >= B >= C > 0, A > C */
    int32_t j1max;           /* 0..8                                                         */
    double bconst2;          /* molecule 2 (linear rotor) constant (hartree)                  */
    int32_t n_j2;            /* 1..8 values of j2                                            */
    int32_t j2[8];           /* each 0..8                                                    */
    double mu;               /* reduced mass (electron masses)                               */
    int32_t n_terms;         /* 1..64                                                        */
    int32_t lam1[64], mu1[64], lam2[64], lam[64];  /* 0 <= mu1 <= lam1 <= 8, lam2 <= 8, triangle */
    double coef[64];         /* hartree */
    double beta[64];         /* 1/bohr  */
    double c6, rd;
    int32_t n_grid;
    double r_min, r_max;
    int32_t path, precision;
} mqct_molmol_params;

/* Build the description of the asymmetric top + linear rotor system above (host arrays released by
 * mqct_free_desc; G in triplet form).  Host-only.  Errors: MQCT_ERR_INVALID_ARG (ranges above, a term
 * outside the triangle |lam1 - lam2| <= lam <= lam1 + lam2), MQCT_ERR_OOM. */
mqct_status mqct_build_molmol(const mqct_molmol_params *p, mqct_system_desc *out);

/* Free the arrays allocated by mqct_build_diatom / mqct_build_asym_top and zero *desc. */
void mqct_free_desc(mqct_system_desc *desc);

/* Validate `desc`, build the spline tables (Sec. III) and coupling layouts of Eq. 12 in
 * device memory and return an immutable system (safe to use from several streams).
 * Validation: N >= 1; finite energies, equal within a level; levels in [0, N); G real
 * symmetric within 1e-12 max|G| and zero between different m (Eq. 6); n_grid >= 4;
 * r_max > r_min; mu > 0; path and precision known; flags 0 or MQCT_PRESCRIBED_TRAJ (the latter
 * with precision MQCT_FP64 only, else MQCT_ERR_UNSUPPORTED).
 * Errors: MQCT_ERR_INVALID_ARG, MQCT_ERR_UNSUPPORTED, MQCT_ERR_OOM, MQCT_ERR_CUDA. */
mqct_status mqct_create_system(const mqct_system_desc *desc, mqct_system *out);
mqct_status mqct_destroy_system(mqct_system sys);
mqct_status mqct_system_info(mqct_system sys, mqct_system_info_t *out);

/* Propagate n trajectories (Eqs. 4-10, RK4); trajectories may refer to different systems
 * (uneven basis sizes), which must share path and precision (see mqct_propagate_ex for how
 * each precision schedules them).
 *   trajs      [n] mqct_traj (host or device)
 *   final_pop  [n][N_t] |a_s|^2 in the caller's state order of the trajectory's system,
 *              rows packed with stride N_max = max over the systems used (the entries past
 *              N_t of a row are not written); or NULL
 *   final_amp  [n][N_max][2] final interaction-picture amplitudes (re, im); or NULL
 *   diag       [n] mqct_diag; or NULL
 * Work order: trajectories are claimed from a device work queue, longest estimated
 * first.  Scratch memory is taken with stream-ordered allocation on `cuda_stream`.
 * With device output pointers the FP64 and FP32 calls only enqueue work and return MQCT_OK;
 * the BF16X3 path synchronises the stream between chunks of 16 steps (it checks on the host
 * whether trajectories are still running), and BF16X3 calls with several systems synchronise
 * it once to size the per-system launches.  With any host
 * output the call synchronises the stream and returns MQCT_ERR_TRAJ if a trajectory status
 * is non-zero.  Errors: MQCT_ERR_INVALID_ARG, MQCT_ERR_UNSUPPORTED, MQCT_ERR_OOM,
 * MQCT_ERR_CUDA, MQCT_ERR_TRAJ. */
mqct_status mqct_propagate(const mqct_system *systems, int32_t n_systems, const mqct_traj *trajs, int32_t n,
                           double *final_pop, double *final_amp, mqct_diag *diag, void *cuda_stream);

/* Options of mqct_propagate_ex; zero-initialise and set what is needed.  None of them changes
 * the arithmetic of a trajectory: they select launch shapes and report timing. */
typedef struct {
    int64_t *t_start_ns;  /* [n] GPU global-timer value (ns) when each trajectory was started, or NULL;
                             host or device pointer                                               */
    int64_t *t_done_ns;   /* [n] GPU global-timer value (ns) when its results were written, or NULL */
    const int32_t *batch_shape; /* [n_systems] HOST array or NULL: shape of the FP32 batched kernel.
                             The call runs one launch for all its systems, whose shape is the first
                             non-zero entry; 0 everywhere = automatic (of the shapes every system
                             fits, the one with the most slots on the GPU that leaves two
                             trajectories per slot, else the one with the fewest slots; the
                             (8,512) and (4,256) shapes first on ties).  1..7 = (slots per CTA at
                             most, threads) of
                             (32,512) (16,512) (8,256) (8,512) (4,512) (16,256) (4,256); each system
                             gets the widest slot count (32, 16, 8 or 4, at most the shape's) its
                             basis fits; a shape that some system does not fit
                             -> MQCT_ERR_UNSUPPORTED                                             */
    const int32_t *tc_slots;    /* [n_systems] HOST array or NULL: trajectories in flight per system
                             on the stage-synchronous paths -- BF16X3: rounded up to a multiple
                             of 64, at most 8192, 0 = automatic (one or two waves of the GPU);
                             FP32 PLAIN: rounded up to a multiple of 32, at most 8192, 0 = every
                             trajectory up to 4096                                              */
} mqct_propagate_opts;

/* mqct_propagate with options (opts may be NULL).  Uneven batches: the trajectories of several
 * systems of one call run together -- FP64: in one persistent launch (each CTA takes the system
 * of the trajectory it claims); FP32: in one persistent launch (up to 16 systems per launch),
 * whose CTAs bind to a system on the device -- at the start in proportion to the systems'
 * estimated work, later to the system with the most work left once theirs is exhausted;
 * BF16X3: one system after the other.  Errors as for mqct_propagate, plus MQCT_ERR_INVALID_ARG
 * for out-of-range options. */
mqct_status mqct_propagate_ex(const mqct_system *systems, int32_t n_systems, const mqct_traj *trajs, int32_t n,
                              double *final_pop, double *final_amp, mqct_diag *diag, const mqct_propagate_opts *opts,
                              void *cuda_stream);

/* mqct_propagate without any memory allocation.  The paper has no counterpart: this call
 * exists for callers that may not allocate GPU memory while they run it -- frameworks that
 * own a fixed device pool and forbid cudaMalloc / cudaFree after start-up, real-time loops
 * that cannot afford allocation latency, processes that must not grow the driver's pool.
 * It runs the same FP64 persistent kernel as mqct_propagate (FP64 systems, plain or
 * factorised) and allocates nothing: its scratch (work-queue counter, system views) is a
 * file-scope device array of 256 + 16 * sizeof(system view) bytes that every GPU loading
 * the library holds until the process exits.
 *   - at most 16 systems per call (the size of that array); more -> MQCT_ERR_INVALID_ARG;
 *   - trajs, final_pop, final_amp and diag must be DEVICE pointers (outputs may be NULL);
 *     layouts as for mqct_propagate; trajectories are claimed in the caller's order;
 *   - the call only enqueues work on `cuda_stream` (two launches: one writes the system views,
 *     which travel by value in its launch parameters, into the array and clears the counter;
 *     the other propagates) and returns MQCT_OK; per-trajectory status is in diag;
 *   - all calls share the one scratch array: two calls whose work overlaps on the GPU (on
 *     different streams, or from different threads without ordering) race on it;
 *   - the first call in a CUDA context (per device, with that device current) looks up the
 *     array's device address; make that first call before any stream capture.  The address is
 *     cached per context: a context created later on the device (e.g. after cudaDeviceReset)
 *     gets its own lookup on its first call.
 * Errors: MQCT_ERR_INVALID_ARG, MQCT_ERR_UNSUPPORTED, MQCT_ERR_CUDA. */
mqct_status mqct_propagate_noalloc(const mqct_system *systems, int32_t n_systems, const mqct_traj *trajs, int32_t n,
                                   double *final_pop, double *final_amp, mqct_diag *diag, void *cuda_stream);

/* Cross sections (Sec. II):
 *   sigma_out[g][l''] = sum_{t : group[t] = g} weight[t] * sum_{s in level l''} final_pop[t][s]
 * final_pop [n][N] (row stride N of `sys`), weight [n], group [n] (entries outside
 * [0, n_groups) are skipped), sigma_out [n_groups][n_levels].  The weight carries the
 * impact-parameter quadrature (e.g. 2 pi b db) and the 1/g average over initial states;
 * a zero weight excludes a trajectory.  Device-side reduction in FP64.  Errors:
 * MQCT_ERR_INVALID_ARG, MQCT_ERR_OOM, MQCT_ERR_CUDA. */
mqct_status mqct_cross_sections(mqct_system sys, const double *final_pop, const double *weight, const int32_t *group,
                                int32_t n, int32_t n_groups, double *sigma_out, void *cuda_stream);

/* Symmetrised cross sections and Maxwell-Boltzmann rate coefficients (Sec. III).
 *
 * Eq. 20, for every pair of levels (a, b) and every computed energy U_k:
 *   sigma_sym[k][a][b] = ( g_a sigma[k][a][b] + g_b sigma[k][b][a] ) / 2,
 * with sigma[k][a][b] = sigma_{a->b}(U_k) (bohr^2) and g the rotational degeneracy of Eq. 19
 * (2j+1 for an atom + rotor).  sigma_sym is symmetric in (a, b).
 *
 * Rates of both directions of every pair (the paper defers the integration to its ref. [44];
 * the readings taken here):
 *   k_{a->b}(T) = (8/(pi mu))^(1/2) (kT)^(-3/2) exp(-(E_b - E_a)/(2 kT)) / g_a
 *                 * integral_{u0}^inf sigma~_ab(U) U exp(-U/kT) dU,
 * U being the mean of the incoming and outgoing translational energies, so that
 * g_a k_{a->b} = g_b k_{b->a} exp(-(E_b - E_a)/kT) exactly.  sigma~_ab(U) is the natural cubic
 * spline through (U_k, sigma_sym[k][a][b]) (negative values taken as zero); below U_1 it falls
 * linearly to zero at the threshold u0 = |E_b - E_a|/2 (or the spline is cut at u0 when
 * u0 >= U_1); above U_K it continues as sigma_sym[K-1] (U/U_K)^p, p the log-log slope of the
 * last two points clipped to [-1, 0].  The finite pieces are integrated by Gauss-Legendre
 * panels no wider than 4 kT (relative error below ~1e-13), the tail in closed form.
 *
 * sigma [K][L][L] (host or device); sigma_sym [K][L][L] output, or NULL to skip it;
 * rate [n_temps][L][L] output, rate[t][a][b] = k_{a->b}(T_t) in bohr^3 per atomic unit of time
 * (x 6.126e-9 for cm^3/s).  The descriptor's arrays are host memory.  Every pair of levels is
 * processed: sigma must hold both directions of each pair whose rates are used.  Outputs in
 * device memory are written asynchronously on `cuda_stream`; host outputs are complete when the
 * call returns.  Errors: MQCT_ERR_INVALID_ARG (sizes, non-increasing or non-positive U, kT <= 0,
 * g <= 0, mu <= 0, reserved != 0, device arrays in the descriptor), MQCT_ERR_OOM, MQCT_ERR_CUDA. */
#define MQCT_RATE_MAX_ENERGIES 32
#define MQCT_RATE_MAX_TEMPS 256
typedef struct {
    int32_t n_levels;            /* L >= 1                                                    */
    int32_t n_energies;          /* K, 2 <= K <= MQCT_RATE_MAX_ENERGIES                       */
    int32_t n_temps;             /* 1 <= n_temps <= MQCT_RATE_MAX_TEMPS                       */
    int32_t reserved;            /* must be 0                                                 */
    double mu;                   /* reduced mass (electron masses), > 0                       */
    const double *u;             /* [K] U_k (hartree), 0 < U_1 < ... < U_K                    */
    const double *kT;            /* [n_temps] k_B T (hartree), > 0                            */
    const double *level_energy;  /* [L] E_l (hartree)                                         */
    const double *degeneracy;    /* [L] g_l > 0                                               */
} mqct_rate_desc;

mqct_status mqct_rate_coefficients(const mqct_rate_desc *desc, const double *sigma, double *sigma_sym, double *rate,
                                   void *cuda_stream);

/* Vector-Jacobian product of the cross sections with respect to the P parameters whose
 * tables were given at create time:
 *   dL_dparam[p] = sum_{g,l''} dL_dsigma[g][l''] * d sigma[g][l''] / d theta_p,
 * by a discrete adjoint of the same RK4 map (the number of steps of every trajectory is
 * held at its forward value), recomputing the forward pass from checkpoints taken every
 * `ckpt` steps.  Arguments as for mqct_propagate / mqct_cross_sections; dL_dsigma
 * [n_groups][n_levels]; dL_dparam [P].  Single system, factorised path, P <= 128, L <= 64.
 * Precision follows the system: MQCT_FP64 -> amplitudes and cotangents in FP64; MQCT_FP32 or
 * MQCT_BF16X3 -> the mixed adjoint: FP32 amplitudes, contraction and cotangents (the step update
 * compensated), phase arguments as fixed-point turn counts, FP64 classical motion, classical
 * cotangents and parameter gradient.  Work vectors live in shared memory when they fit (N up to
 * ~800 in FP64, ~1500 in FP32), else in global memory.  Errors: MQCT_ERR_INVALID_ARG,
 * MQCT_ERR_UNSUPPORTED (no parameter tables, plain path, prescribed trajectories, limits above),
 * MQCT_ERR_OOM, MQCT_ERR_CUDA, MQCT_ERR_TRAJ. */
mqct_status mqct_adjoint(mqct_system sys, const mqct_traj *trajs, int32_t n, const double *weight,
                         const int32_t *group, int32_t n_groups, const double *dL_dsigma, int32_t ckpt,
                         double *dL_dparam, void *cuda_stream);

/* Thread-local message describing the last failure of a call on this thread. */
const char *mqct_last_error(void);

/* Number of this library's kernel launches made by the last mqct_propagate, mqct_propagate_ex,
 * mqct_propagate_noalloc, mqct_cross_sections, mqct_adjoint or mqct_rate_coefficients call on
 * this thread (reset at the start of each of these calls).  Kernels of a CUDA graph that the call
 * runs are counted once per execution (the number of chunks a graph's loop ran is read back from
 * the device); kernels of other libraries the call uses (CUB's sort and select) are not counted.
 * Calls that return asynchronously have issued all their launches when they return. */
int64_t mqct_last_launch_count(void);

/* Library version string. */
const char *mqct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MQCT_H */

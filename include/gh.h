/*
 * gh.h -- C ABI of libgh: the generalized-harmonic (GH) right-hand side on
 * spherical-shell spectral subdomains, with RK4, filters and boundary
 * handling, on one NVIDIA GB300 (sm_103a), in FP64.
 *
 * Method: Lewis & Pfeiffer, "GPU-Accelerated Simulations of Isolated Black
 * Holes" (arXiv:1804.09101).  The paper fixes the structure: collocation data
 * on I1 x S2 shells expanded in T_k(r) Y_lm (Sec. 3.4), derivatives as cached
 * linear maps (Sec. 3.4, Eqs. Differentiation and DifferentiatorI1S2), the
 * DiffJac contraction (Sec. 3.3, Eq. DiffJac), the filters (Sec. 3.4), the GH
 * equations and the three boundary cases (Sec. 3.5 and Sec. 5), and analytic
 * Kerr-Schild data of mass m and spin chi (Sec. 3.1).  The GH equations are
 * the standard first-order system of Lindblom et al. (2006).
 *
 * Conventions shared by every call
 *  - All arrays passed to the library are DEVICE pointers to FP64 data on the
 *    current CUDA device unless a parameter says "host".  The caller owns them;
 *    the library never frees or retains them past the call.
 *  - A state vector holds, for each shell in creation order, the array
 *    u[r][field][theta][phi] (phi fastest): n_r * 50 * (L+1) * 2(L+1) doubles.
 *    Field order: psi_ab = p, Pi_ab = 10+p, Phi_iab = 20+10i+p, where
 *    p enumerates (ab) = 00,01,02,03,11,12,13,22,23,33 and i = x,y,z.
 *  - Grid of a shell: r at the n_r Chebyshev-Gauss-Lobatto points of
 *    [r_in, r_out] (ascending), theta at the L+1 Gauss-Legendre points
 *    (ascending), phi_k = 2 pi k / (2(L+1)).  Cartesian coordinates are the
 *    Kerr-Schild x, y, z of a hole at the origin with spin along +z.
 *  - Every call is enqueued on the domain's CUDA stream (gh_set_stream) and
 *    returns without synchronising, except where stated.  Errors raised on the
 *    device (a non-finite constraint norm) are latched and reported by
 *    gh_sync.  No call throws or aborts; each returns a gh_status, and
 *    gh_last_error gives a one-line reason.
 *  - Errors common to every call, unless its comment says more: GH_EINVAL for
 *    a NULL domain or a NULL required pointer, GH_ECUDA when a CUDA call or a
 *    launch fails (the reason in gh_last_error).  Device-side errors are only
 *    read by gh_sync, so that no other call has to synchronise.
 */
#ifndef GH_H
#define GH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GH_OK = 0,
  GH_EINVAL = 1,      /* invalid argument (shape, pointer, parameter)          */
  GH_ENOMEM = 2,      /* device allocation failed                              */
  GH_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed           */
  GH_ETIMEOUT = 4,    /* a bounded device-side wait ran out                    */
  GH_ENONFINITE = 5,  /* a constraint norm came out NaN or Inf                 */
  GH_ENOTSUP = 6      /* not supported by this library for these settings     */
} gh_status;

/* One spherical shell: r in [r_in, r_out], n_r radial points, harmonics l <= L,
 * belonging to black hole bh (0, 1, ...).  Requires 0 < r_in < r_out,
 * 3 <= n_r <= 64, 1 <= L <= 47.  The shells of one hole are consecutive in the
 * array, ordered by radius, and adjacent (r_in of the next == r_out of the
 * previous) with equal L; holes are independent of one another (the paper's
 * one-domain-per-process picture, Sec. 4, batched into one set of launches). */
typedef struct {
  double r_in, r_out;
  int n_r, L;
  int bh;
} gh_shell;

/* Evolution parameters.
 * gamma0, gamma1, gamma2: GH constraint-damping parameters (Lindblom et al.).
 * filt_alpha, filt_order: exponential Chebyshev filter sigma_k =
 *   exp(-alpha (k/(n_r-1))^order) applied along r when radial_filter_on != 0
 *   (the paper's ExpCheb filter, Sec. 3.4).
 * sh_keep_l: Heaviside filter in l (keep l <= sh_keep_l) on every shell, -1 for
 *   none, or -2 for floor(2L/3) of each shell (the paper's Heaviside filter,
 *   Sec. 3.4; applied per component). */
typedef struct {
  double gamma0, gamma1, gamma2;
  double filt_alpha;
  int filt_order;
  int radial_filter_on;
  int sh_keep_l;
} gh_params;

typedef struct gh_domain gh_domain;

/* Create a domain of n_shells shells around one or more independent holes
 * (see gh_shell for the ordering rules).  Builds the cached
 * operator matrices on the host in FP64 (the paper's matrix dictionary,
 * Sec. 3.4) and uploads them together with grid tables; allocates the
 * library's own scratch (three derivative buffers of one state each plus
 * small tables).  stream: a cudaStream_t or NULL for the legacy stream.
 * Errors: GH_EINVAL for invalid shells or params, GH_ENOMEM, GH_ECUDA.
 * The domain starts with zero gauge source and a flat (Minkowski) boundary
 * background; call gh_set_analytic_kerr_schild or gh_set_gauge and
 * gh_set_background before evolving. */
gh_status gh_create_domain(const gh_shell* shells, int n_shells, const gh_params* params,
                           void* stream, gh_domain** out);

/* Free everything the domain owns.  Synchronises its stream first. */
gh_status gh_destroy_domain(gh_domain* dom);

/* Change the stream later calls are enqueued on. */
gh_status gh_set_stream(gh_domain* dom, void* stream);

/* on = 1 (the default): each right-hand side runs its radial derivative map
 * on a second stream the domain owns, beside the angular maps on the domain's
 * stream, forked and joined by events.  Both read the state and write separate
 * buffers, so the results are bitwise the same as with on = 0, where the maps
 * run one after the other.  Calls still behave as if everything ran on the
 * domain's stream, and graph captures include the fork and join.  With the
 * profiler on (gh_profile_enable) the maps run one after the other so that
 * each family is timed alone.  Errors: GH_EINVAL unless on is 0 or 1. */
gh_status gh_set_overlap(gh_domain* dom, int on);

/* Sizes in doubles: one state vector; one RK4 work area (gh_rk4_step). */
long long gh_state_size(const gh_domain* dom);
long long gh_num_points(const gh_domain* dom);
long long gh_rk4_work_size(const gh_domain* dom);
int gh_num_shells(const gh_domain* dom);

/* Write the exact Kerr-Schild state of hole bh (mass M, dimensionless spin chi
 * along +z, a = chi M) into the shells of that hole in u (device, one state),
 * and set, on those shells, the gauge source H_a = -Gamma_a, d_i H_a of that
 * solution and the boundary background used by the characteristic boundary
 * conditions.  bh = -1: every shell of the domain.  Kerr-Schild data: Sec. 3.1
 * (Eq. dimensionlessspin).  Computed on the device with forward-mode
 * second-order dual numbers. */
gh_status gh_set_analytic_kerr_schild(gh_domain* dom, int bh, double M, double chi, double* u);
/* The same for a dimensionless spin vector chi[3] of any direction (host
 * pointer), a = chi M: the paper's own test hole has chi = (0.2, 0.3, 0.4)
 * (Sec. 3.1, Eq. dimensionlessspin).  With a.x the Euclidean dot product and
 * a x x the cross product: H = M r^3 / (r^4 + (a.x)^2), l_0 = 1,
 * l_i = (r x_i - (a x x)_i + (a.x) a_i / r) / (r^2 + a^2),
 * r^2 = (R^2 - a^2)/2 + sqrt((R^2 - a^2)^2/4 + (a.x)^2).  GH_EINVAL unless
 * M > 0 and |chi| < 1. */
gh_status gh_set_analytic_kerr_schild_spin(gh_domain* dom, int bh, double M, const double chi[3], double* u);

/* Scale the time step of hole bh: its shells advance by dt * scale in every
 * gh_rk4_step(dom, dt, ...).  Lets holes of different resolution take their
 * own stable steps inside one batched step.  Default 1. */
gh_status gh_set_dt_scale(gh_domain* dom, int bh, double scale);

/* Replace the gauge source: H (device) holds, for each shell, [r][4][theta][phi]
 * with H_a; dH (device) holds [r][12][theta][phi] with entry 4*i + a = d_i H_a.
 * d_t H_a = 0 always. */
gh_status gh_set_gauge(gh_domain* dom, const double* H, const double* dH);

/* Copy the domain's gauge source out, in the layout gh_set_gauge takes. */
gh_status gh_get_gauge(const gh_domain* dom, double* H, double* dH);

/* Take the boundary background (lapse, shift, unit normal used by the
 * characteristic projection) from the metric part of state u_bg (device). */
gh_status gh_set_background(gh_domain* dom, const double* u_bg);

/* Add a perturbation to u (device).  kind 0: ingoing Gaussian shell on psi,
 * dpsi_ab = A exp(-(R-Rc)^2/w^2) sum c_lm Y_lm on all 10 components, with
 * dPhi_iab = d_i dpsi_ab and dPi_ab = -(d_R dpsi - beta^k d_k dpsi)/alpha from
 * the boundary background's source metric (the current Kerr-Schild hole).
 * kind 1: dPi_ab = exp(-((R-Rc)/w)^2) sum c_lm Y_lm on all 10 components
 * (A ignored).  coeffs (host) holds (lmax+1)^2 real Y_lm coefficients in the
 * order l = 0..lmax, m = -l..l; Y_lm real orthonormal, sqrt(2) cos(m phi) for
 * m > 0 and sqrt(2) sin(|m| phi) for m < 0. */
gh_status gh_add_perturbation(gh_domain* dom, int kind, double A, double Rc, double w,
                              int lmax, const double* coeffs, double* u);

/* Cartesian derivatives d_i u of all 50 fields: du (device) holds 3 states,
 * du[i * state_size + ...].  Radial and angular derivative maps (Eq.
 * DifferentiatorI1S2) followed by the DiffJac contraction (Eq. DiffJac). */
gh_status gh_derivatives(gh_domain* dom, const double* u, double* du);

/* One right-hand side evaluation dudt = F(u): derivatives, the pointwise GH
 * equations (GHEqns) and the boundary conditions (ApplyBCs): outer boundary
 * freezes the incoming characteristic fields, internal boundaries exchange
 * incoming characteristic time derivatives upwind, the excision boundary is a
 * no-op (Sec. 5).  u and dudt must not overlap. */
gh_status gh_rhs(gh_domain* dom, const double* u, double* dudt);

/* One classic RK4 step of size dt on u (device, in place), followed by the
 * filters the domain's params switch on.  work (device) must hold
 * gh_rk4_work_size doubles.  If norm2_pre (device, nullable) is given, the
 * constraint norm of the incoming u is written to norm2_pre[s] for each shell
 * s (computed inside the first stage, from the same derivatives). */
gh_status gh_rk4_step(gh_domain* dom, double dt, double* u, double* work, double* norm2_pre);

/* The same RK4 steps for data in HOST memory: copies u_in (host, one state)
 * to a device state the domain owns (allocated on the first call, with an RK4
 * work area), takes n_steps gh_rk4_step steps (filters included), copies the
 * result to u_out (host, one state; may equal u_in) and, if norm2_out (host,
 * n_shells doubles) is given, the constraint norms of the state the last step
 * started from.  The steps replay a CUDA graph of one step on those buffers,
 * captured on the first call with a given dt (and norm2_out null or not) and
 * again after any setter that changes the step's launches (algorithm,
 * schedule, overlap, frame, outer condition, S2 filter); it is separate from
 * gh_rk4_graph_capture's graph.  Synchronises the stream before returning.
 * Pinned host buffers (cudaHostAlloc, cudaHostRegister) copy asynchronously at
 * full speed; pageable ones work too.  With n_steps == 1, both buffers pinned
 * and at least one filter on, no separate copies run: the step's first radial
 * derivative reads u_in over the host link (writing the device state as it
 * goes) and its last filter writes u_out, so the transfers overlap those
 * kernels' arithmetic; that form is captured once per (dt, norm2_out null or
 * not, u_in, u_out) and gives the same bits as the copy form.  The domain's
 * filters run SH truncation first, then the radial filter (they commute).
 * Errors: GH_EINVAL for n_steps < 1 or a NULL buffer, GH_ENOMEM on the first
 * call, GH_ECUDA. */
gh_status gh_rk4_step_host(gh_domain* dom, double dt, int n_steps, const double* u_in, double* u_out,
                           double* norm2_out);

/* CUDA graph of one RK4 step: gh_rk4_graph_capture records the launches of
 * gh_rk4_step(dom, dt, u, work, norm2_pre) (same pointers, profiler off) into a
 * graph owned by the domain, replacing any previous one; nothing runs.
 * gh_rk4_graph_launch replays it n_steps times on the domain's stream, which
 * removes the per-launch host overhead of the many small launches of a step. */
gh_status gh_rk4_graph_capture(gh_domain* dom, double dt, double* u, double* work, double* norm2_pre);
gh_status gh_rk4_graph_launch(gh_domain* dom, int n_steps);

/* Apply the domain's filters to u (device) in place; work as for gh_rk4_step. */
gh_status gh_apply_filters(gh_domain* dom, double* u, double* work);

/* Constraints of u: c_out (device, nullable) receives, per shell,
 * [r][64][theta][phi] with C_a (0..3), C_iab = d_i psi_ab - Phi_iab (4+10i+p) and
 * C_ijab = d_i Phi_jab - d_j Phi_iab for (ij) = xy,xz,yz (34+10q+p);
 * norm2 (device) receives per shell sum_points w dV sum_c C_c^2 with the
 * Clenshaw-Curtis x Gauss-Legendre x uniform quadrature. */
gh_status gh_constraints(gh_domain* dom, const double* u, double* c_out, double* norm2);

/* gh_rhs_noalloc: the same right-hand side as gh_rhs, computed without any
 * device allocation.  The three derivative work buffers come from one fixed
 * array inside the library (3 x 2^20 doubles = 24 MiB, present on every GPU
 * that loads the library until the process exits) instead of the domain's
 * own scratch.  It is meant for callers that must not allocate GPU memory at
 * call time: a host whose own memory pool owns the device memory, or a
 * time-critical loop that cannot afford an allocation or the synchronisation
 * it can bring.  The domain itself is still created (and allocated) once, up
 * front.  The paper has no counterpart of this entry point.
 *   - Limit: gh_state_size(dom) <= 2^20 doubles (about 20,000 grid points);
 *     larger domains get GH_EINVAL with a message.  Use gh_rhs for them.
 *   - The first call on each device looks up the array's device address with
 *     that device current; make this first call before any stream capture.
 *     The address is kept for the life of the process, so a device reset
 *     (cudaDeviceReset, or the primary context torn down) while the library
 *     is loaded is not supported for this entry point.
 *   - Every call uses the same array: calls that run at the same time on the
 *     GPU (other streams, other host threads) race and corrupt each other's
 *     results.  Serialise them.
 *   - Nothing in the array needs to start at zero: each call writes every
 *     element it later reads. */
gh_status gh_rhs_noalloc(gh_domain* dom, const double* u, double* dudt);

/* ---------------------------------------------------------------- adjoint
 * Vector-Jacobian products of the evolution (reverse-mode derivatives), for
 * gradients of functionals of the evolved state.  The angular maps are
 * transposed with the algorithm the domain uses: the folded separable maps
 * (the default) with the forward's tables read with input and output
 * swapped, the plain separable maps with their transposed plans; the dense
 * traced matrices have no transpose here (GH_ENOTSUP).  The boundary projection is linear
 * in dudt (fixed background) and the filters and derivative maps are linear,
 * so the adjoint is exact up to rounding: transposed boundary conditions, the
 * reverse pass of the pointwise GH algebra, transposed DiffJac, radial and
 * angular maps (Eqs. DiffJac and DifferentiatorI1S2, transposed). */

/* ubar += (dF/du)^T kbar for F = gh_rhs; u, kbar, ubar: device states. */
gh_status gh_rhs_vjp(gh_domain* dom, const double* u, const double* kbar, double* ubar);

/* ubar_n = (d step / d u_n)^T ubar_np1 for step = gh_rk4_step(dom, dt, .) with
 * its filters; u_n is the state the step started from.  Recomputes the stage
 * states and keeps their spherical derivatives for the reverse pass.  work:
 * gh_rk4_vjp_work_size doubles (device; 16 states).  ubar_n must not alias
 * ubar_np1. */
long long gh_rk4_vjp_work_size(const gh_domain* dom);
gh_status gh_rk4_step_vjp(gh_domain* dom, double dt, const double* u_n, const double* ubar_np1,
                          double* ubar_n, double* work);

/* The same step with its three intermediate stage states (u_n + dt/2 k1,
 * u_n + dt/2 k2, u_n + dt k3) written to stages (3 states, device), and the
 * step VJP that reuses them instead of recomputing them.  The latter also adds
 * cweight * d/du (sum of the shells' constraint norms) at u_n to ubar_n, which
 * shares the derivative passes with the last stage (0: no such term). */
gh_status gh_rk4_step_save(gh_domain* dom, double dt, double* u, double* work, double* norm2_pre,
                           double* stages);
gh_status gh_rk4_step_vjp_saved(gh_domain* dom, double dt, const double* u_n, const double* stages,
                                const double* ubar_np1, double* ubar_n, double* work, double cweight);

/* ubar += weight * d/du (sum over shells of the constraint norm that
 * gh_constraints writes to norm2). */
gh_status gh_constraint_energy_vjp(gh_domain* dom, const double* u, double weight, double* ubar);

/* grad[lm] (host, (lmax+1)^2 doubles) = <ubar, d u / d c_lm> for the Pi-mode
 * perturbation of gh_add_perturbation (kind 1 only; lmax <= 8).  Synchronises. */
gh_status gh_perturbation_vjp(gh_domain* dom, int kind, double Rc, double w, int lmax, const double* ubar,
                              double* grad);

/* Block until the domain's stream is idle; returns the first latched device
 * error (GH_ENONFINITE) or GH_ECUDA, then clears the latch. */
gh_status gh_sync(gh_domain* dom);

/* Last error message of this domain (or of the last failed gh_create_domain
 * when dom is NULL).  Valid until the next call on the same domain. */
const char* gh_last_error(const gh_domain* dom);

/* Number of kernel launches the library has enqueued on this domain so far. */
long long gh_launch_count(const gh_domain* dom);

/* How the angular maps (d/dtheta, d/dphi and the SH filter) are evaluated.
 * GH_ALG_DENSE: one dense (N_theta N_phi)^2 matrix per map, the paper's traced
 *   matrices of Eq. DifferentiatorI1S2 (built on first selection).
 * GH_ALG_SEPARABLE: the same linear maps factorised as a phi DFT, one
 *   N_theta x N_theta Legendre map per Fourier mode, and an inverse DFT; equal
 *   to the dense maps up to rounding, with far fewer flops.
 * GH_ALG_SEPARABLE_FOLDED (default): the separable maps with the cos/sin
 *   symmetries of the uniform phi grid and the equatorial parity of Pbar_lm
 *   folded out (about 3x fewer flops again); any L (odd N_theta: the equator
 *   ring is its own mirror; N_phi % 4 == 2: no quarter point is). */
enum { GH_ALG_DENSE = 0, GH_ALG_SEPARABLE = 1, GH_ALG_SEPARABLE_FOLDED = 2 };
gh_status gh_set_algorithm(gh_domain* dom, int algorithm);

/* Rotating dual frame (Sec. 3.1: collocation points fixed in grid
 * coordinates, equations in inertial coordinates, related by a time-dependent
 * map; Sec. 3.3: SpatialCoordJac).  The map is the rigid rotation
 * x = R(t) x_grid about `axis` (host pointer, any nonzero length) at rate
 * omega (0: static grid, the default).  The evolved values are inertial-frame
 * components at the grid points, so every right-hand side becomes
 *   d/dt u = ApplyBCs(F(u, R d_grid u)) + xdot^k (R d_grid u)_k,
 *   xdot = omega e x (R x_grid):
 * the map's Jacobian on the derivative index (after DiffJac), the boundary
 * conditions on the inertial rate F, and the grid-velocity term.  The
 * background must be invariant under rotations about the axis (Schwarzschild:
 * any axis; Kerr: its spin axis): its gauge source and boundary background at
 * a moving point are then the stored t = 0 values with rotated components, and
 * the characteristic speeds do not change (xdot is tangential).
 * gh_rhs, gh_constraints and gh_derivatives evaluate at the domain's time
 * (gh_set_time / gh_get_time); gh_rk4_step and accepted gh_dp5_step attempts
 * advance it and use their stage times.  The clock also lives on the device
 * and each step computes its stage frames from it there, so a captured RK4
 * graph replays with the live time (each gh_rk4_graph_launch of n steps
 * advances the clock by n dt).  The adjoint entry points evaluate at the
 * clock too (gh_rk4_step_vjp: the clock is the time of u_n; the step's stage
 * times follow from it), with the rotated DiffJac, gauge source and boundary
 * background transposed and the grid-velocity term's transpose added.  With
 * omega != 0, steps and adjoint calls on domains with a dt scale other than 1
 * return GH_ENOTSUP (one clock per domain).
 * gh_set_rotating_frame and gh_set_time synchronise the stream;
 * gh_set_rotating_frame discards a captured graph; GH_EINVAL for a zero axis
 * or a non-finite rate. */
gh_status gh_set_rotating_frame(gh_domain* dom, const double axis[3], double omega);
/* gh_set_frame_map: the general time-dependent map of the dual frame (Sec. 3.1:
 * grid and inertial coordinates share the time and are related by a
 * time-dependent map), x = a(t) R(t) x_grid + T(t) with a(t) = 1 + adot t
 * (expansion, or contraction for adot < 0), R(t) the rotation about axis by
 * omega t, T(t) = V t (translation); t is the domain clock (gh_set_time).  The
 * derivative index takes the map's Jacobian, d_inertial = R d_grid / a (the
 * SpatialCoordJac of Sec. 3.3), each RHS adds xdot . d u after the boundary
 * conditions, and the hole's gauge source and the boundary background are
 * evaluated at the moving inertial points every stage (so every hole must
 * have been set with gh_set_analytic_kerr_schild*; GH_EINVAL otherwise), the
 * boundary being the moving sphere |x - T| = a r with its characteristic speeds
 * taken relative to it.  axis: 3 numbers (host), not all zero; rates finite.
 * Replaces gh_set_rotating_frame's rotation (which rotates the stored gauge
 * source and needs a background symmetric about the axis); the adjoint entry
 * points return GH_ENOTSUP under a general map.  Captured RK4 graphs replay
 * with the live clock. */
gh_status gh_set_frame_map(gh_domain* dom, const double axis[3], double omega, double adot, const double V[3]);

gh_status gh_set_time(gh_domain* dom, double t);
gh_status gh_get_time(const gh_domain* dom, double* t);

/* Outer boundary condition (ApplyBCs at the external boundary, Sec. 5).
 * GH_BC_FREEZE (default): incoming characteristic time derivatives set to 0.
 * GH_BC_CONSTRAINT_PRESERVING: Bjorhus form for the u^psi and u^0 families --
 *   at incoming points d_t u^psi_ab = D_t u^psi_ab + v_psi n^i C_iab and
 *   d_t u^0_iab = D_t u^0_iab + v_0 P_i^k n^j C_jkab (D_t: the characteristic
 *   projection of the equations, C_iab = d_i psi_ab - Phi_iab, C_jkab = d_j Phi_kab
 *   - d_k Phi_jab), which removes the incoming normal derivative of those fields;
 *   u^- is frozen.  The adjoint entry points transpose these terms (they are
 *   linear in u and its derivatives for the fixed background).
 * GH_BC_CONSTRAINT_PRESERVING_FULL: as GH_BC_CONSTRAINT_PRESERVING, and u^-
 *   no longer frozen: the gauge constraint C_a = H_a + Gamma_a may not enter.
 *   Its incoming characteristic field, K_a = (d_t C_a - beta^i d_i C_a) / N
 *   + n^i d_i C_a (its derivative along the outgoing null direction;
 *   background N, beta, n), holds the normal derivative of u^-; in Bjorhus
 *   form that normal derivative is replaced in the u^- equation by the value
 *   for which K_a, with the interior equations, vanishes.  d_t u^- is taken in
 *   the span of the l l, l m and transverse-trace parts of the background null
 *   tetrad (l = (t + n)/sqrt 2), with its gauge and transverse-traceless parts
 *   frozen: one 5x5 solve per outer point (a singular system leaves u^-
 *   frozen there).  Static grid only: GH_ENOTSUP with a rotating frame or a
 *   general map (set either way round).  The adjoint entry points transpose
 *   it, nonlinear in u as it is (the inverse metric, the lapse and the solve),
 *   with one extra interior right-hand side per reverse RHS.
 * Synchronises the stream and discards a captured RK4 graph. */
enum { GH_BC_FREEZE = 0, GH_BC_CONSTRAINT_PRESERVING = 1, GH_BC_CONSTRAINT_PRESERVING_FULL = 2 };
gh_status gh_set_outer_bc(gh_domain* dom, int mode);

/* Angular (S2) filter mode (Sec. 3.1: the filter acts on tensors through
 * tensor spherical harmonics; Sec. 3.4: its matrix couples the components).
 * GH_SH_FILTER_COMPONENT (default): every one of the 50 fields is truncated to
 *   Y_lm, l <= keep, on its own (Cartesian components treated as scalars).
 * GH_SH_FILTER_TENSOR: each spatial tensor (psi_00, psi_0i, psi_ij, the same
 *   for Pi, Phi_i00, Phi_i0j, Phi_ijk) is written in the local complex frame
 *   r_hat, m = (theta_hat + i phi_hat)/sqrt(2), conj(m); a frame component of
 *   spin weight s (#m - #conj(m)) is projected onto the spin-weighted
 *   harmonics sY_lm, |s| <= l <= keep, and the tensor is rebuilt with the dual
 *   frame.  keep is the domain's sh_keep_l (per shell for -2).  Uses a device
 *   buffer of 62 doubles per grid point (the 31 independent complex frame
 *   components), allocated by the first switch to this mode on a domain with
 *   an angular filter (GH_ECUDA if it does not fit).  The adjoint entry points use the filter's transpose (the
 *   spin projection is self-adjoint under the quadrature weights).
 *   Synchronises the stream and discards a captured RK4 graph; GH_EINVAL for
 *   an unknown mode. */
enum { GH_SH_FILTER_COMPONENT = 0, GH_SH_FILTER_TENSOR = 1 };
gh_status gh_set_sh_filter(gh_domain* dom, int mode);

/* Dormand-Prince 5(4) adaptive step: the paper's time stepper (Sec. 2.1; the
 * embedded pair of Dormand & Prince 1980, seven right-hand sides per attempt,
 * no stage reused across steps).  One attempt from u with step dt:
 *   k_s = F(u + dt sum_j a_sj k_j) (F = gh_rhs, boundary conditions included),
 *   unew = u + dt sum_j b_j k_j (fifth order),
 *   err = sqrt(mean over every value of (e / (atol + rtol max(|u|, |unew|)))^2)
 *   with e = dt sum_j (b_j - bhat_j) k_j (fourth-order companion).
 * accepted = (err <= 1); then u <- unew followed by the filters (as for RK4),
 * else u is left unchanged.  dt_next = dt min(5, max(0.2, 0.9 err^(-1/5)))
 * (5 dt when err = 0).  err_out, accepted and dt_next are host pointers; the
 * call synchronises the stream to read err.  work: device scratch of
 * gh_dp5_work_size doubles (the seven stage derivatives and two states).
 * GH_EINVAL for dt <= 0, negative tolerances or both zero; GH_ENOTSUP when a
 * shell has a dt scale other than 1 (gh_set_dt_scale). */
long long gh_dp5_work_size(const gh_domain* dom);
gh_status gh_dp5_step(gh_domain* dom, double dt, double rtol, double atol, double* u, double* work,
                      double* err_out, int* accepted, double* dt_next);

/* Work-schedule autotuner.  The schedule is how the radial and folded angular
 * maps split their work (the paper has no counterpart: its traced-matrix
 * products run as library GEMMs, Sec. 3.4); it never changes the arithmetic of
 * any output of the forward maps, so every schedule of sched[0..7] gives
 * bitwise identical results.
 *   sched[0], sched[1]: radial derivative (folded: the centro-antisymmetric
 *     CGL matrix applied through the ceil(n_r/2) rows that give a mirror pair
 *     of outputs each) -- FMA chains per pass (2..4) and row groups per
 *     column (1..4, one grid row each);
 *   sched[2], sched[3]: the same for the radial ExpCheb filter;
 *   sched[4], sched[5]: folded d/dtheta, d/dphi kernel -- threads per block
 *     (32..512, a multiple of 32) and the shared-memory budget per block in
 *     bytes (8 KiB..200 KiB), which sets the rows per block of every shell
 *     (for shells with N_phi = 16, 32, 64 these set the Legendre stage; their
 *     ring FFTs run in fixed blocks of 128 threads);
 *   sched[6], sched[7]: the same for the folded SH filter;
 *   sched[8]: reverse pass of the pointwise algebra (gh_rhs_vjp and the step
 *     VJPs) with one thread per point (0) or ten, one per symmetric pair (1):
 *     the pair-split form does ~3x the work with a ~3x shorter serial path per
 *     thread and wins on small grids (default: 1 up to 8,192 points); not
 *     timed by gh_autotune.  Results agree to rounding, not bitwise.
 * gh_autotune times every candidate of each map on this domain (CUDA events
 * on the domain's stream, one warm-up and `reps` timed launches each, the
 * domain's own scratch as input and output), keeps the fastest, and
 * synchronises the stream.  gh_set_schedule validates and installs a
 * schedule (GH_EINVAL otherwise).  Both discard a captured RK4 graph
 * (capture again).  n must be at least GH_SCHEDULE_LEN. */
#define GH_SCHEDULE_LEN 9
gh_status gh_autotune(gh_domain* dom, int reps);
gh_status gh_get_schedule(const gh_domain* dom, int* sched, int n);
gh_status gh_set_schedule(gh_domain* dom, const int* sched, int n);

/* Kernel families for the profiler below. */
typedef enum {
  GH_K_RADIAL = 0,        /* radial derivative map (Chebyshev, folded n_r x n_r)   */
  GH_K_ANGULAR = 1,       /* angular derivative maps (d/dtheta, d/dphi)             */
  GH_K_POINTWISE = 2,     /* fused DiffJac + GH right-hand side + RK4 combine       */
  GH_K_BC = 3,            /* characteristic boundary conditions                     */
  GH_K_RADIAL_FILTER = 4, /* exponential Chebyshev filter                          */
  GH_K_ANGULAR_FILTER = 5,/* spherical-harmonic truncation filter                   */
  GH_K_REDUCE = 6,        /* constraint-norm reduction                              */
  GH_K_COMBINE = 7,       /* Dormand-Prince stage combinations and error norm       */
  GH_K_FAMILIES = 8
} gh_kernel_family;

/* Profiler: while enabled, every kernel the domain launches is bracketed by
 * CUDA events recorded on the domain's stream.  gh_profile_read synchronises
 * the stream, adds the elapsed times of all completed brackets of one family
 * to *total_ms and their number to *launches, and clears that family. */
gh_status gh_profile_enable(gh_domain* dom, int on);
gh_status gh_profile_read(gh_domain* dom, int family, double* total_ms, long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* GH_H */

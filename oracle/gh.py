"""First-order generalized-harmonic (GH) system: RHS, constraints, boundaries (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper names the GH evolution equations ("GHEqns", Sec. 3.1 and Sec. 3.5)
and the three boundary cases (Sec. 5: characteristic data exchanged at
internal boundaries, conditions at the outer boundary, nothing at the
excision boundary) without printing them.  The equations below are the
standard first-order GH system (Lindblom, Scheel, Kidder, Owen & Rinne 2006),
restated from the mathematics; the boundary treatment is the simplified
characteristic one documented in ``rhs_with_boundaries``.

Per point the 50 evolved fields are psi_ab (10), Pi_ab (10) and Phi_iab (30),
symmetric pairs packed in the order (00,01,02,03,11,12,13,22,23,33):
field index psi = p, Pi = 10 + p, Phi_i = 20 + 10 i + p.

All pointwise functions take arrays with arbitrary leading (point) axes and
trailing tensor axes, and are written with einsum index strings that mirror
the equations term by term.
"""
import numpy as np

PAIRS = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
NF = 50


# ----------------------------------------------------------------- packing
def unpack_fields(u):
    """u[..., 50] -> psi[..., 4, 4], Pi[..., 4, 4], Phi[..., 3, 4, 4]."""
    shp = u.shape[:-1]
    psi = np.zeros(shp + (4, 4))
    Pi = np.zeros(shp + (4, 4))
    Phi = np.zeros(shp + (3, 4, 4))
    for p, (a, b) in enumerate(PAIRS):
        psi[..., a, b] = psi[..., b, a] = u[..., p]
        Pi[..., a, b] = Pi[..., b, a] = u[..., 10 + p]
        for i in range(3):
            Phi[..., i, a, b] = Phi[..., i, b, a] = u[..., 20 + 10 * i + p]
    return psi, Pi, Phi


def pack_fields(psi, Pi, Phi):
    """Inverse of unpack_fields (reads the a <= b entries)."""
    shp = psi.shape[:-2]
    u = np.zeros(shp + (50,))
    for p, (a, b) in enumerate(PAIRS):
        u[..., p] = psi[..., a, b]
        u[..., 10 + p] = Pi[..., a, b]
        for i in range(3):
            u[..., 20 + 10 * i + p] = Phi[..., i, a, b]
    return u


# --------------------------------------------------------------- 3+1 split
def spacetime_split(psi):
    """Lapse, shift, spatial inverse metric, normal and inverse spacetime metric.

    g_ij = psi_ij, g^ij its inverse, beta_i = psi_0i, beta^i = g^ij beta_j,
    alpha = sqrt(beta^i beta_i - psi_00), t^a = (1, -beta^i)/alpha,
    t_a = (-alpha, 0, 0, 0), psi^ab = g^ab-with-shift: psi^00 = -1/alpha^2,
    psi^0i = beta^i/alpha^2, psi^ij = g^ij - beta^i beta^j/alpha^2, and the
    spatial projector g^i_a = delta^i_a + t^i t_a.
    """
    g = psi[..., 1:, 1:]
    ginv = np.linalg.inv(g)
    beta_dn = psi[..., 0, 1:]
    beta_up = np.einsum("...ij,...j->...i", ginv, beta_dn)
    alpha = np.sqrt(np.einsum("...i,...i->...", beta_up, beta_dn) - psi[..., 0, 0])
    shp = alpha.shape
    t_up = np.zeros(shp + (4,))
    t_up[..., 0] = 1.0 / alpha
    t_up[..., 1:] = -beta_up / alpha[..., None]
    t_dn = np.zeros(shp + (4,))
    t_dn[..., 0] = -alpha
    psi_inv = np.zeros(shp + (4, 4))
    a2 = alpha * alpha
    psi_inv[..., 0, 0] = -1.0 / a2
    psi_inv[..., 0, 1:] = beta_up / a2[..., None]
    psi_inv[..., 1:, 0] = beta_up / a2[..., None]
    psi_inv[..., 1:, 1:] = ginv - np.einsum("...i,...j->...ij", beta_up, beta_up) / a2[..., None, None]
    proj = np.zeros(shp + (3, 4))                     # g^i_a
    for i in range(3):
        proj[..., i, 1 + i] = 1.0
    proj = proj + np.einsum("...i,...a->...ia", t_up[..., 1:], t_dn)
    return dict(ginv=ginv, beta_dn=beta_dn, beta_up=beta_up, alpha=alpha,
                t_up=t_up, t_dn=t_dn, psi_inv=psi_inv, proj=proj)


def christoffel_first_kind(s, Pi, Phi):
    """d_c psi_ab = t_c Pi_ab + g^i_c Phi_iab and Gamma_abc = (d_b psi_ac + d_c psi_ab - d_a psi_bc)/2."""
    d = (np.einsum("...c,...ab->...cab", s["t_dn"], Pi)
         + np.einsum("...ic,...iab->...cab", s["proj"], Phi))
    Gam = 0.5 * (np.einsum("...bac->...abc", d) + np.einsum("...cab->...abc", d)
                 - np.einsum("...abc->...abc", d))
    return d, Gam


def gauge_constraint(s, Gam, H):
    """C_a = H_a + Gamma_a, Gamma_a = psi^bc Gamma_abc."""
    return H + np.einsum("...bc,...abc->...a", s["psi_inv"], Gam)


# ---------------------------------------------------------- GH right-hand side
def gh_rhs_pointwise(u, du, H, dH, gamma0, gamma1, gamma2):
    """Time derivative of the 50 GH fields at each point.

    u[..., 50]; du[..., 3, 50] = d_k u (Cartesian); H[..., 4] = H_a;
    dH[..., 3, 4] = d_i H_a (d_t H_a = 0).  Returns dudt[..., 50].

    d_t psi_ab = (1+g1) b^k d_k psi_ab - N Pi_ab - g1 b^i Phi_iab
    d_t Pi_ab  = b^k d_k Pi_ab - N g^ki d_k Phi_iab + g1 g2 b^k d_k psi_ab
                 + 2N psi^cd (g^ij Phi_ica Phi_jdb - Pi_ca Pi_db - psi^ef Gam_ace Gam_bdf)
                 - 2N nabla_(a H_b) - N/2 t^c t^d Pi_cd Pi_ab - N t^c Pi_ci g^ij Phi_jab
                 + N g0 (2 delta^c_(a t_b) - psi_ab t^c) C_c - g1 g2 b^i Phi_iab
    d_t Phi_iab = b^k d_k Phi_iab - N d_i Pi_ab + N g2 d_i psi_ab
                 + N/2 t^c t^d Phi_icd Pi_ab + N g^jk t^c Phi_ijc Phi_kab - N g2 Phi_iab
    with N = alpha, b = beta, nabla_a H_b = d_a H_b - psi^cd Gam_dab H_c.
    """
    psi, Pi, Phi = unpack_fields(u)
    dpsi, dPi, dPhi = unpack_fields(du)              # dpsi[...,k,a,b], dPhi[...,k,i,a,b]
    s = spacetime_split(psi)
    N = s["alpha"]
    b_up = s["beta_up"]
    ginv = s["ginv"]
    t_up, t_dn = s["t_up"], s["t_dn"]
    psi_inv = s["psi_inv"]
    _, Gam = christoffel_first_kind(s, Pi, Phi)
    C = gauge_constraint(s, Gam, H)

    shp = N.shape
    dH4 = np.zeros(shp + (4, 4))                     # d_a H_b, d_0 H_b = 0
    dH4[..., 1:, :] = dH
    Gam_up = np.einsum("...cd,...dab->...cab", psi_inv, Gam)
    nablaH = dH4 - np.einsum("...cab,...c->...ab", Gam_up, H)
    nablaH_sym = 0.5 * (nablaH + np.einsum("...ab->...ba", nablaH))

    Nb = N[..., None, None]
    Ni = N[..., None, None, None]

    dt_psi = ((1.0 + gamma1) * np.einsum("...k,...kab->...ab", b_up, dpsi)
              - Nb * Pi
              - gamma1 * np.einsum("...i,...iab->...ab", b_up, Phi))

    quad = (np.einsum("...cd,...ij,...ica,...jdb->...ab", psi_inv, ginv, Phi, Phi)
            - np.einsum("...cd,...ca,...db->...ab", psi_inv, Pi, Pi)
            - np.einsum("...cd,...ef,...ace,...bdf->...ab", psi_inv, psi_inv, Gam, Gam))
    tPt = np.einsum("...c,...d,...cd->...", t_up, t_up, Pi)
    tPi_i = np.einsum("...c,...ci->...i", t_up, Pi[..., :, 1:])
    tC = np.einsum("...c,...c->...", t_up, C)
    damp = (np.einsum("...b,...a->...ab", t_dn, C) + np.einsum("...a,...b->...ab", t_dn, C)
            - psi * tC[..., None, None])
    dt_Pi = (np.einsum("...k,...kab->...ab", b_up, dPi)
             - Nb * np.einsum("...ki,...kiab->...ab", ginv, dPhi)
             + gamma1 * gamma2 * np.einsum("...k,...kab->...ab", b_up, dpsi)
             + 2.0 * Nb * quad
             - 2.0 * Nb * nablaH_sym
             - 0.5 * Nb * tPt[..., None, None] * Pi
             - Nb * np.einsum("...i,...ij,...jab->...ab", tPi_i, ginv, Phi)
             + gamma0 * Nb * damp
             - gamma1 * gamma2 * np.einsum("...i,...iab->...ab", b_up, Phi))

    tPhit = np.einsum("...c,...d,...icd->...i", t_up, t_up, Phi)
    dt_Phi = (np.einsum("...k,...kiab->...iab", b_up, dPhi)
              - Ni * dPi
              + gamma2 * Ni * dpsi
              + 0.5 * Ni * np.einsum("...i,...ab->...iab", tPhit, Pi)
              + Ni * np.einsum("...jk,...c,...ijc,...kab->...iab", ginv, t_up, Phi[..., :, 1:, :], Phi)
              - gamma2 * Ni * Phi)
    return pack_fields(dt_psi, dt_Pi, dt_Phi)


# --------------------------------------------------------------- constraints
def constraints_pointwise(u, du, H):
    """The 64 stored constraint components per point.

    [0:4]   C_a = H_a + Gamma_a
    [4:34]  C_iab = d_i psi_ab - Phi_iab   (index 4 + 10 i + p)
    [34:64] C_ijab = d_i Phi_jab - d_j Phi_iab for (i,j) = (x,y),(x,z),(y,z)
            (index 34 + 10 q + p)
    """
    psi, Pi, Phi = unpack_fields(u)
    dpsi, dPi, dPhi = unpack_fields(du)
    s = spacetime_split(psi)
    _, Gam = christoffel_first_kind(s, Pi, Phi)
    C = gauge_constraint(s, Gam, H)
    shp = C.shape[:-1]
    out = np.zeros(shp + (64,))
    out[..., 0:4] = C
    C3 = dpsi - Phi
    C4 = np.einsum("...ijab->...ijab", dPhi) - np.einsum("...jiab->...ijab", dPhi)
    for p, (a, b) in enumerate(PAIRS):
        for i in range(3):
            out[..., 4 + 10 * i + p] = C3[..., i, a, b]
        for q, (i, j) in enumerate([(0, 1), (0, 2), (1, 2)]):
            out[..., 34 + 10 * q + p] = C4[..., i, j, a, b]
    return out


def gauge_constraint_derivative(u, v, H, w):
    """Directional derivative of C_a = H_a + psi^bc Gamma_abc along (v, w).

    u[..., 50] is the state, v[..., 50] a direction in field space (a time
    derivative or a Cartesian derivative d_i u), H[..., 4] the gauge source and
    w[..., 4] its derivative along the same direction.  The product rule,
    term by term (a prime is the derivative along v):
      psi'^ab = -psi^ac psi'_cd psi^db,
      N = (-psi^00)^(-1/2)          ->  N' = N^3 psi'^00 / 2,
      t_c = (-N, 0, 0, 0)           ->  t'_c = (-N', 0, 0, 0),
      t^i = -N psi^0i               ->  t'^i = -N' psi^0i - N psi'^0i,
      g^i_c = delta^i_c + t^i t_c   ->  g'^i_c = t'^i t_c + t^i t'_c,
      d_c psi_ab = t_c Pi_ab + g^i_c Phi_iab, and its prime from the above,
      C'_a = w_a + psi'^bc Gamma_abc + psi^bc Gamma'_abc,
    with Gamma'_abc built from the primed d_c psi_ab as Gamma_abc is from d_c psi_ab.
    """
    psi, Pi, Phi = unpack_fields(u)
    dpsi, dPi, dPhi = unpack_fields(v)
    s = spacetime_split(psi)
    psi_inv = s["psi_inv"]
    N = s["alpha"]
    dpsi_inv = -np.einsum("...ac,...cd,...db->...ab", psi_inv, dpsi, psi_inv)
    dN = 0.5 * N ** 3 * dpsi_inv[..., 0, 0]
    dt_dn = np.zeros(N.shape + (4,))
    dt_dn[..., 0] = -dN
    t_up_i = s["t_up"][..., 1:]
    dt_up_i = -dN[..., None] * psi_inv[..., 0, 1:] - N[..., None] * dpsi_inv[..., 0, 1:]
    dproj = (np.einsum("...i,...c->...ic", dt_up_i, s["t_dn"])
             + np.einsum("...i,...c->...ic", t_up_i, dt_dn))
    _, Gam = christoffel_first_kind(s, Pi, Phi)
    dd = (np.einsum("...c,...ab->...cab", dt_dn, Pi) + np.einsum("...c,...ab->...cab", s["t_dn"], dPi)
          + np.einsum("...ic,...iab->...cab", dproj, Phi) + np.einsum("...ic,...iab->...cab", s["proj"], dPhi))
    dGam = 0.5 * (np.einsum("...bac->...abc", dd) + np.einsum("...cab->...abc", dd)
                  - np.einsum("...abc->...abc", dd))
    return (w + np.einsum("...bc,...abc->...a", dpsi_inv, Gam)
            + np.einsum("...bc,...abc->...a", psi_inv, dGam))


def boundary_tetrad(bg):
    """Null vectors and transverse projector of the background at boundary points.

    From the background lapse N, shift beta^i, spatial metric g_ij and unit
    normal n_i (n^i = g^ij n_j): the unit normal t^a = (1, -beta^i)/N,
    t_a = (-N, 0, 0, 0); the spacetime normal n^a = (0, n^i),
    n_a = (beta^i n_i, n_i); the outgoing null vector l = (t + n)/sqrt(2)
    (both index positions), the incoming k = (t - n)/sqrt(2), and the
    projector onto the 2-surface orthogonal to both,
    P_ab = psi_ab + t_a t_b - n_a n_b, with the background 4-metric psi_ab.
    """
    N, beta, g, n_dn, n_up = bg["alpha"], bg["beta_up"], bg["g_dn"], bg["n_dn"], bg["n_up"]
    shp = N.shape
    beta_dn = np.einsum("...ij,...j->...i", g, beta)
    psi4 = np.zeros(shp + (4, 4))
    psi4[..., 0, 0] = -N * N + np.einsum("...i,...i->...", beta, beta_dn)
    psi4[..., 0, 1:] = beta_dn
    psi4[..., 1:, 0] = beta_dn
    psi4[..., 1:, 1:] = g
    t_dn = np.zeros(shp + (4,))
    t_dn[..., 0] = -N
    t_up = np.zeros(shp + (4,))
    t_up[..., 0] = 1.0 / N
    t_up[..., 1:] = -beta / N[..., None]
    n4_dn = np.zeros(shp + (4,))
    n4_dn[..., 0] = np.einsum("...i,...i->...", beta, n_dn)
    n4_dn[..., 1:] = n_dn
    n4_up = np.zeros(shp + (4,))
    n4_up[..., 1:] = n_up
    r2 = np.sqrt(0.5)
    P = psi4 + np.einsum("...a,...b->...ab", t_dn, t_dn) - np.einsum("...a,...b->...ab", n4_dn, n4_dn)
    return dict(l_dn=r2 * (t_dn + n4_dn), l_up=r2 * (t_up + n4_up), k_dn=r2 * (t_dn - n4_dn),
                k_up=r2 * (t_up - n4_up), P=P)


def uminus_constraint_part(dudt0, dudt_int, u_b, du_b, H_b, dH_b, bg, gamma2):
    """The u^- time derivative of the constraint-preserving outer condition.

    Reading of the condition on u^- (the paper's outer boundary is constraint
    preserving, Sec. 5; the GH literature splits u^- into constraint, physical
    and gauge parts): the gauge constraint C_a may not enter through the
    boundary.  C_a propagates like a wave, whose incoming characteristic field
    is its derivative along the outgoing null direction (as u^- = Pi - n.Phi is
    -(t + n).d psi for psi):
        K_a = (t^c + n^c) d_c C_a = (d_t C_a - beta^i d_i C_a) / N + n^i d_i C_a.
    Evaluated with the interior equations it holds the normal derivative of
    u^- as 2 B(d_n u^-), B the linear map from a u^- derivative to d_t C_a / N
    (a u^- derivative S changes Pi by S/2 and Phi_i by -n_i S/2, from_char).
    In the Bjorhus form the condition replaces that normal derivative in the
    u^- equation, d_t u^- = -v_- d_n u^- + ..., by the value for which K_a,
    with the interior equations, vanishes:
        d_t u^- = D_t u^- + (v_- / 2) B^-1 K_a[interior],   v_- = -n.beta - N,
    so the boundary equation of u^- no longer holds its own normal derivative.
    In terms of K_a[w] taken along a time derivative whose u^- part is w
    (K_a is affine in w, with slope B): B(S) = -K_a[0] + (N - n.beta)/(2N) K_a[D_t u^-],
    where the normal-derivative parts of the two terms cancel.  (Zeroing K_a
    along the corrected time derivative instead leaves -N d_n u^- in the
    boundary equation, upwinded against the incoming direction; along the
    incoming null direction, (t - n).d C_a, it restates the interior equation.)

    S is sought in the 4-dimensional subspace
        S_ab = l_a lam_b + lam_a l_b + sig P_ab,   l^b lam_b = 0
    (the l l, l m and transverse-trace parts in a null tetrad (l, k, m, conj m)),
    on which B is invertible; the remaining six (k k, k m, l k: gauge; the
    transverse traceless part: physical) lie in the kernel of B and stay frozen
    at zero.  Four conditions and l^b lam_b = 0 fix (lam, sig).

    dudt0[..., 50] and dudt_int[..., 50] are the time derivative with the other
    families' conditions applied and w^- = 0, resp. w^- = D_t u^- (interior);
    u_b, du_b[..., 3, 50] the state and its Cartesian derivatives; H_b[..., 4],
    dH_b[..., 3, 4] the gauge source and its derivatives; bg the boundary
    background (N, beta, n).  Returns S[..., 4, 4].
    """
    tet = boundary_tetrad(bg)
    N, beta, n_up = bg["alpha"], bg["beta_up"], bg["n_up"]
    shp = N.shape
    zero4 = np.zeros(shp + (4,))
    dC = np.stack([gauge_constraint_derivative(u_b, du_b[..., i, :], H_b, dH_b[..., i, :]) for i in range(3)],
                  axis=-2)                                                     # [..., i, a]

    def K(dudt):
        dtC = gauge_constraint_derivative(u_b, dudt, H_b, zero4)
        return ((dtC - np.einsum("...i,...ia->...a", beta, dC)) / N[..., None]
                + np.einsum("...i,...ia->...a", n_up, dC))

    nb = np.einsum("...i,...i->...", bg["n_dn"], beta)
    target = -K(dudt0) + ((N - nb) / (2.0 * N))[..., None] * K(dudt_int)
    l = tet["l_dn"]
    eye = np.eye(4)
    basis = [np.einsum("...a,c->...ac", l, eye[b]) + np.einsum("a,...c->...ac", eye[b], l) for b in range(4)]
    basis.append(tet["P"])
    z44 = np.zeros(shp + (4, 4))
    z344 = np.zeros(shp + (3, 4, 4))
    M = np.zeros(shp + (5, 5))
    rhs_v = np.zeros(shp + (5,))
    for j, E in enumerate(basis):
        v = from_char(z44, z344, z44, E, bg, gamma2)
        M[..., 0:4, j] = gauge_constraint_derivative(u_b, v, H_b, zero4) / N[..., None]
    M[..., 4, 0:4] = tet["l_up"]
    rhs_v[..., 0:4] = target
    x = np.linalg.solve(M, rhs_v[..., None])[..., 0]
    lam, sig = x[..., 0:4], x[..., 4]
    return (np.einsum("...a,...b->...ab", l, lam) + np.einsum("...a,...b->...ab", lam, l)
            + sig[..., None, None] * tet["P"])


# ---------------------------------------------------- characteristic fields
def boundary_background(psi_bg, X, Y, Z):
    """Unit normal and speeds data from the background metric at boundary points.

    n_i = d_i R / |d R|_g with R the Euclidean radius, n^i = g^ij n_j.
    Returns dict with n_dn[...,3], n_up[...,3], alpha, beta_up[...,3] and the
    spatial metric g_dn[...,3,3].
    """
    s = spacetime_split(psi_bg)
    R = np.sqrt(X * X + Y * Y + Z * Z)
    dR = np.stack([X / R, Y / R, Z / R], axis=-1)
    norm = np.sqrt(np.einsum("...ij,...i,...j->...", s["ginv"], dR, dR))
    n_dn = dR / norm[..., None]
    n_up = np.einsum("...ij,...j->...i", s["ginv"], n_dn)
    return dict(n_dn=n_dn, n_up=n_up, alpha=s["alpha"], beta_up=s["beta_up"], g_dn=psi_bg[..., 1:, 1:].copy())


def char_speeds(bg, gamma1):
    """Speeds (v_psi, v_0, v_plus, v_minus) along n = +R direction.

    A boundary that moves with the grid (a time-dependent map) carries
    bg["n_xdot"] = n_i xdot^i, the normal grid velocity; the speeds relative
    to the moving boundary are the inertial ones minus it (every family's
    advection gains the grid velocity in the grid frame)."""
    nb = np.einsum("...i,...i->...", bg["n_dn"], bg["beta_up"])
    sh = bg.get("n_xdot", 0.0)
    return (-(1.0 + gamma1) * nb - sh, -nb - sh, -nb + bg["alpha"] - sh, -nb - bg["alpha"] - sh)


def to_char(v, bg, gamma2):
    """Characteristic projection of a field vector v[..., 50].

    w_psi = psi, w_0_iab = P_i^k Phi_kab (P_i^k = delta_i^k - n_i n^k),
    w_pm = Pi +- n^k Phi_kab - gamma2 psi.
    """
    psi, Pi, Phi = unpack_fields(v)
    nPhi = np.einsum("...k,...kab->...ab", bg["n_up"], Phi)
    w0 = Phi - np.einsum("...i,...ab->...iab", bg["n_dn"], nPhi)
    wp = Pi + nPhi - gamma2 * psi
    wm = Pi - nPhi - gamma2 * psi
    return psi, w0, wp, wm


def from_char(wpsi, w0, wp, wm, bg, gamma2):
    """Inverse of to_char: psi = w_psi, Pi = (w+ + w-)/2 + gamma2 w_psi,
    Phi_iab = n_i (w+ - w-)/2 + w_0_iab."""
    psi = wpsi
    Pi = 0.5 * (wp + wm) + gamma2 * wpsi
    Phi = np.einsum("...i,...ab->...iab", bg["n_dn"], 0.5 * (wp - wm)) + w0
    return pack_fields(psi, Pi, Phi)


def apply_outer_bc(dudt_b, bg, gamma1, gamma2):
    """Freezing condition: incoming (v < 0) characteristic time derivatives set to 0."""
    w = list(to_char(dudt_b, bg, gamma2))
    for q, v in enumerate(char_speeds(bg, gamma1)):
        mask = (v < 0.0)
        w[q] = np.where(mask.reshape(mask.shape + (1,) * (w[q].ndim - mask.ndim)), 0.0, w[q])
    return from_char(*w, bg, gamma2)


def apply_outer_bc_cp(dudt_b, u_b, du_b, bg, gamma1, gamma2, H_b=None, dH_b=None):
    """Constraint-preserving outer condition of Bjorhus form for the u^psi and
    u^0 families; for u^- freezing, or (H_b and dH_b given) the constraint
    part of uminus_constraint_part with its gauge and physical parts frozen;
    u^+ frozen if it were incoming.

    The outer boundary condition of the paper is constraint preserving (Sec. 5);
    its equations are those of the standard first-order GH system (Lindblom
    et al. 2006, Sec. VI).  For the two families whose incoming parts carry the
    derivative constraints, the characteristic time derivative computed from
    the equations, D_t w, is replaced at incoming points by
        d_t w_psi_ab  = D_t w_psi_ab + v_psi n^i C_iab,        C_iab  = d_i psi_ab - Phi_iab,
        d_t w_0_iab   = D_t w_0_iab  + v_0 P_i^k n^j C_jkab,   C_jkab = d_j Phi_kab - d_k Phi_jab,
    which removes the incoming normal derivative of the field from its
    evolution equation.  u_b[..., 50] is the state and du_b[..., 3, 50] its
    Cartesian derivatives at the boundary points.
    """
    wpsi, w0, wp, wm = to_char(dudt_b, bg, gamma2)
    v_psi, v_0, v_p, v_m = char_speeds(bg, gamma1)
    psi, Pi, Phi = unpack_fields(u_b)
    dpsi = np.stack([unpack_fields(du_b[..., i, :])[0] for i in range(3)], axis=-3)   # [..., i, a, b]
    dPhi = np.stack([unpack_fields(du_b[..., j, :])[2] for j in range(3)], axis=-4)   # [..., j, k, a, b]
    C3 = dpsi - Phi
    C4 = dPhi - np.swapaxes(dPhi, -4, -3)
    nC3 = np.einsum("...i,...iab->...ab", bg["n_up"], C3)
    m = np.einsum("...j,...jkab->...kab", bg["n_up"], C4)
    Pm = m - np.einsum("...i,...k,...kab->...iab", bg["n_dn"], bg["n_up"], m)
    inc_psi = (v_psi < 0.0)[..., None, None]
    inc_0 = (v_0 < 0.0)[..., None, None, None]
    wpsi = np.where(inc_psi, wpsi + v_psi[..., None, None] * nC3, wpsi)
    w0 = np.where(inc_0, w0 + v_0[..., None, None, None] * Pm, w0)
    wp = np.where((v_p < 0.0)[..., None, None], 0.0, wp)
    inc_m = (v_m < 0.0)[..., None, None]
    if H_b is None:
        wm = np.where(inc_m, 0.0, wm)
    else:
        dudt0 = from_char(wpsi, w0, wp, np.zeros_like(wm), bg, gamma2)
        dudt_i = from_char(wpsi, w0, wp, wm, bg, gamma2)
        wm = np.where(inc_m, uminus_constraint_part(dudt0, dudt_i, u_b, du_b, H_b, dH_b, bg, gamma2), wm)
    return from_char(wpsi, w0, wp, wm, bg, gamma2)


def apply_interface_bc(dudt_in, dudt_out, bg, gamma1, gamma2):
    """Upwind exchange at a shared radius between an inner and an outer shell.

    With n along +R: a field with v < 0 travels inward, so both sides take the
    outer shell's value; v > 0: both take the inner shell's; v == 0: each keeps
    its own.  Returns the new (dudt_in, dudt_out) boundary slices.
    """
    wi = list(to_char(dudt_in, bg, gamma2))
    wo = list(to_char(dudt_out, bg, gamma2))
    for q, v in enumerate(char_speeds(bg, gamma1)):
        shp = v.shape + (1,) * (wi[q].ndim - v.ndim)
        neg = (v < 0.0).reshape(shp)
        pos = (v > 0.0).reshape(shp)
        new_i = np.where(neg, wo[q], wi[q])
        new_o = np.where(pos, wi[q], wo[q])
        wi[q], wo[q] = new_i, new_o
    return from_char(*wi, bg, gamma2), from_char(*wo, bg, gamma2)

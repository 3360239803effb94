/*
 * pflb_oracle.c -- plain FP64 CPU oracle of the conservative Allen-Cahn
 * phase-field lattice Boltzmann step (D3Q19) with the local mobility
 * correction, the filtered hydrodynamic collision, the mu*grad(phi) force
 * from central-difference stencils, and the wettability (contact-angle) and
 * free-slip friction conditions at solid voxels.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the package's smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, table or helper with the CUDA path.
 *
 * Layout (deliberately unlike the GPU path): array of cells, h[cell*19+i],
 * two buffers, push streaming.  Every quantity is double.  Cells are indexed
 * x fastest: cell = x + nx*(y + ny*z).  The box is periodic in x, y and z;
 * walls are solid voxels.
 *
 * Notation follows the paper: h_i are the phase-field populations (Eq. 1),
 * g_i (the paper's g-bar) the hydrodynamic populations (Eq. 5).  T = 1/3.
 *
 * Readings of passages the paper leaves open, the same on both sides of the
 * parity tests:
 *   R1  rho = rho_L + phi*(rho_H - rho_L), rho_dif = rho_H - rho_L, phi=1 heavy.
 *   R2  Filtered collision (Eqs. 9-11): G_eq = E + K/2 with
 *       E_i = rho*Gamma_i + w_i*(P/T - rho); non-equilibrium = g - g_eq
 *       (g_eq of Eq. 6); Pi = sum_l c_l c_l (g_l - g_eq_l), full tensor.
 *   R3  Per-step order: phi -> wall ghosts -> stencils -> macros -> collide
 *       -> stream; u in h_eq is the same step's hydrodynamic velocity.
 *   R4  "Delta phi" in delta-theta is the CD Laplacian; s = lap/(|lap|+eps),
 *       a sign of the Laplacian regularised by eps.  Printed literally,
 *       lap/|lap+eps| divides by zero at lap = -eps (the pole that eps is
 *       said to avoid) and leaves [-1, 1] near it; the two agree to eps/|lap|
 *       wherever |lap| >> eps.
 *   R5  n (interface normal) and n_w (wall normal, into the fluid) differ.
 *   R6  phi_smpl = phi of the wall node itself; one ghost per solid link.
 *   R8  If the tangential part of grad(phi) at the wall has norm < 1e-10,
 *       t = 0 and w = -cos(theta) n_w.
 *   R9  w = -cos(theta) n_w + sin(theta) t (rotation of n_w by pi - theta
 *       about n_w x grad(phi)); theta measured inside the phi=1 phase.
 *   R10 artanh argument clamped to [-1+1e-12, 1-1e-12].
 *   R11 Ghost update uses the previous step's ghosts in grad(phi); initial
 *       ghosts equal phi of the wall node.
 *   R12 Hysteresis blend: ghost_n = b*ghost_{n-1} + (1-b)*ghost_new.
 *   R13 h: halfway bounce-back at solid links.
 *   R14 Free-slip band: an edge link of fluid cell x into a flat axis-aligned
 *       wall is specularly reflected onto the tangential neighbour y when
 *       band_lo <= phi <= band_hi at both x and y; otherwise bounce-back.
 *   R16 Initial state: h = h_eq(phi0, u=0, n(grad phi0)), g = g_eq(P0, u=0)
 *       with K from grad phi0, ghosts = phi of the wall node.
 *   R17 Solid cells are never updated; sums run over fluid cells only.
 *   R22 Open x boundaries (Sec. IV A: Dirichlet pressure with Neumann
 *       velocity and phi; velocity inlets): the fluid cells of the planes
 *       x = 0 and x = nx-1 are boundary cells.  At the start of each step a
 *       boundary state (phi_b, P_b, u_b) is formed: given values, and for the
 *       Neumann quantities those of the adjacent interior cell (x = 1 or
 *       nx-2) in their bulk form, phi = sum h, P = T sum g,
 *       rho u = sum c g + F/2.  Pressure boundary: P_b given, phi_b and u_b
 *       from the neighbour.  Velocity boundary: u_b and phi_b given, P_b
 *       from the neighbour.  The boundary cell's phi is phi_b (it enters the
 *       neighbours' stencils); it is not collided: its post-collision
 *       populations are the equilibria h_i = phi_b Gamma_i(u_b),
 *       g_i = w_i P_b / T + rho_b (Gamma_i(u_b) - w_i), streamed as usual
 *       (bounce-back at solid links, no free-slip band, no ghost update).
 *       What streams into a boundary cell (including the periodic wrap
 *       between the two planes) is discarded.  Given values may be ramped
 *       linearly over a number of steps from those in effect (the rest
 *       state P = 0, u = 0 when the boundaries were off).
 *
 *   R23 Sub-voxel walls (Sec. II B's volume-weighted sampling, the offset
 *       walls of Sec. IV A), a light form of the volumetric overlap
 *       weighting: each cell carries a solid volume fraction s (1 on solid
 *       voxels, 0 on plain fluid cells, 0 < s < 1 on fluid cells that the
 *       wall cuts).  Cut cells are fluid cells in every other respect (they
 *       hold populations; bounce-back and the free-slip band act only at
 *       links into solid voxels).  A wall node is a fluid cell with a
 *       neighbour of s > 0; it keeps one ghost phi_{s,i} per link into a
 *       solid voxel and per link into a cut cell that points into the wall.
 *       Its sample phi_smpl averages phi over a parallelepiped one spacing
 *       thick standing on the wall: (1 - s_x) phi(x) + s_x phi(x + c_n),
 *       with c_n the axis direction nearest the wall normal (phi(x) in
 *       place of phi(x + c_n) when that cell is solid).  In the CD stencils
 *       a cut neighbour y = x + c_i along a link into the wall (c_i . n_w
 *       < 0) contributes s_y phi_{s,i} + (1 - s_y) phi(y): the ghost for the
 *       part of y inside the wall, y's own phi for the rest; a link parallel
 *       to the wall or away from it does not cross the wall and takes phi(y).
 *       With every s in {0, 1} this is R6 exactly.
 *
 * Parity unpinned by the paper (pinned only oracle <-> GPU): the sub-step
 * order (R3), the ghost lag (R11), the blend side (R12) and the free-slip
 * band rule (R14).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define TT (1.0 / 3.0) /* lattice temperature T = c_s^2 (Sec. II A) */

/* D3Q19 velocities: rest, +-x, +-y, +-z, then the 12 edge directions in
 * opposite pairs.  Weights are the textbook D3Q19 ones. */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const int OPP[Q] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
static const double WQ[Q] = {1.0 / 3.0,
                             1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

typedef struct {
    double sigma, W, M;           /* surface tension, interface width, mobility */
    double rho_H, rho_L;          /* heavy (phi=1) and light (phi=0) densities */
    double nu_H, nu_L;            /* kinematic viscosities (water, air) */
    double theta_deg;             /* input contact angle when no per-cell angle */
    double Fex[3];                /* external body force */
    double gamma, phi_M, phi_m, D, eps; /* mobility correction constants */
    double blend;                 /* hysteresis blend factor b */
    double band_lo, band_hi;      /* free-slip band on phi */
    double F_tilde, F_width;      /* optimised F(phi) = (tanh((phi-F_tilde)/F_width)+1)/2 */
    int F_mode;                   /* 0: F(phi)=phi, 1: optimised tanh F */
    int mobility_corr;            /* 1: add delta-theta */
    int free_slip;                /* 1: free-slip band at flat walls */
    int nthreads;                 /* OpenMP threads (1 = serial) */
} orc_params;

typedef struct {
    int nx, ny, nz;
    int64_t N;
    orc_params p;
    uint8_t *solid;   /* [N] */
    double *frac;     /* [N] solid volume fraction (R23), NULL: s = solid[] */
    int8_t *cn;       /* [N] axis direction nearest the wall normal (R23) */
    double *nw;       /* [N*3] wall normal into the fluid (wall nodes) */
    double *cth, *sth;/* [N] cos/sin of the input contact angle */
    double *h, *g;    /* [N*Q] current populations (post-stream) */
    double *h2, *g2;  /* [N*Q] streaming targets */
    double *phi;      /* [N] order parameter of the current step */
    double *ghost;    /* [N*Q] phi_{s,i} of wall node x for solid link i */
    double *ghost_old;/* [N*Q] scratch: ghosts of the previous step */
    int bc_type[2];   /* x = 0, x = nx-1: 0 periodic, 1 pressure, 2 velocity (R22) */
    double bc_val[2][5]; /* given P, ux, uy, uz, phi (targets) */
    double bc_from[2][5];/* values at the start of the ramp */
    int64_t bc_t0, bc_ramp; /* ramp start step and length (0: targets at once) */
    double *bstate;   /* [2*ny*nz*5] boundary states phi, P, ux, uy, uz */
    int64_t step;
} orc_lattice;

/* ---------------------------------------------------------------- helpers */

static inline int64_t wrap(int64_t a, int64_t n) { a %= n; return a < 0 ? a + n : a; }

static inline int64_t nbr(const orc_lattice *L, int64_t cell, int i) {
    int64_t x = cell % L->nx, y = (cell / L->nx) % L->ny, z = cell / ((int64_t)L->nx * L->ny);
    x = wrap(x + CX[i], L->nx);
    y = wrap(y + CY[i], L->ny);
    z = wrap(z + CZ[i], L->nz);
    return x + (int64_t)L->nx * (y + (int64_t)L->ny * z);
}

static inline int64_t shift(const orc_lattice *L, int64_t cell, int dx, int dy, int dz) {
    int64_t x = cell % L->nx, y = (cell / L->nx) % L->ny, z = cell / ((int64_t)L->nx * L->ny);
    x = wrap(x + dx, L->nx);
    y = wrap(y + dy, L->ny);
    z = wrap(z + dz, L->nz);
    return x + (int64_t)L->nx * (y + (int64_t)L->ny * z);
}

/* Solid volume fraction of a cell (R23). */
static inline double sfrac(const orc_lattice *L, int64_t cell) {
    return L->solid[cell] ? 1.0 : (L->frac ? L->frac[cell] : 0.0);
}

static inline int is_wall_node(const orc_lattice *L, int64_t cell) {
    if (L->solid[cell]) return 0;
    for (int i = 1; i < Q; ++i)
        if (sfrac(L, nbr(L, cell, i)) > 0.0) return 1;
    return 0;
}

static inline double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* ------------------------------------------------- per-cell model pieces */

/* Gamma_i(u) of Eq. 3. */
void orc_gamma(const double u[3], double G[Q]) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
        G[i] = WQ[i] * (1.0 + cu / TT + cu * cu / (2.0 * TT * TT) - uu / (2.0 * TT));
    }
}

/* CD gradient and Laplacian of Eq. 13 from the 19 neighbour values
 * val[i] = phi(x + c_i) (val[0] = phi(x)).  The gradient's sum runs over
 * all i of (phi(x+c_i) - phi(x-c_i)) c_i w_i / (2T). */
void orc_cd_stencil(const double val[Q], double grad[3], double *lap) {
    double gx = 0, gy = 0, gz = 0, l = 0;
    for (int i = 0; i < Q; ++i) {
        double diff = val[i] - val[OPP[i]];
        gx += diff * CX[i] * WQ[i];
        gy += diff * CY[i] * WQ[i];
        gz += diff * CZ[i] * WQ[i];
        l += (val[i] - val[0]) * WQ[i];
    }
    grad[0] = gx / (2.0 * TT);
    grad[1] = gy / (2.0 * TT);
    grad[2] = gz / (2.0 * TT);
    *lap = 2.0 * l / TT;
}

/* Chemical potential of Eq. 7. */
double orc_chem_pot(const orc_params *p, double phi, double lap) {
    return 48.0 * p->sigma / p->W * phi * (phi - 1.0) * (phi - 0.5) - 1.5 * p->sigma * p->W * lap;
}

/* F(x) = max(0, min(1, x)) and delta-theta of Eq. 4. */
double orc_delta_theta(const orc_params *p, double phi, const double grad[3], double lap) {
    double F1a = clamp01((phi - p->phi_M) / p->D);
    double F1b = clamp01(-(phi - 1.0) / p->D);
    double F2a = clamp01(phi / p->D);
    double F2b = clamp01(-(phi - p->phi_m) / p->D);
    double Y1 = F1a < F1b ? F1a : F1b;
    double Y2 = F2a < F2b ? F2a : F2b;
    double s = lap / (fabs(lap) + p->eps);
    double gnorm = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
    return p->gamma * p->M / (TT * p->W) * gnorm * ((1.0 + s) * Y1 + (1.0 - s) * Y2);
}

/* theta of Eq. 3 (plus the correction when enabled). */
double orc_theta(const orc_params *p, double phi, const double grad[3], double lap) {
    double th = (p->M / TT) * (1.0 - 4.0 * (phi - 0.5) * (phi - 0.5)) / p->W;
    if (p->mobility_corr) th += orc_delta_theta(p, phi, grad, lap);
    return th;
}

/* h equilibrium of Eq. 2: phi*Gamma_i + theta*w_i*(c_i . n), with the
 * interface normal n = grad/(|grad| + eps). */
void orc_h_eq(const orc_params *p, double phi, const double u[3], const double grad[3], double lap,
              double heq[Q]) {
    double G[Q];
    orc_gamma(u, G);
    double gnorm = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
    double n[3] = {grad[0] / (gnorm + p->eps), grad[1] / (gnorm + p->eps), grad[2] / (gnorm + p->eps)};
    double th = orc_theta(p, phi, grad, lap);
    for (int i = 0; i < Q; ++i) {
        double cn = CX[i] * n[0] + CY[i] * n[1] + CZ[i] * n[2];
        heq[i] = phi * G[i] + th * WQ[i] * cn;
    }
}

/* Mixture relaxation time of Eq. 8 with F(phi) = phi (plain) or the
 * optimised tanh F(phi) of Sec. III A; tau = nu/T + 1/2. */
double orc_tau_mix(const orc_params *p, double phi) {
    double Fp = phi;
    if (p->F_mode == 1) Fp = 0.5 * (tanh((phi - p->F_tilde) / p->F_width) + 1.0);
    double tau_w = p->nu_H / TT + 0.5, tau_a = p->nu_L / TT + 0.5;
    return (1.0 - Fp) * tau_a + Fp * tau_w;
}

/* Macroscopic recovery (text after Eq. 11):
 *   rho u = sum_i c_i g_i + (mu grad phi + F_ex)/2,
 *   P     = T sum_i g_i + (T rho_dif / 2) u . grad phi.                */
void orc_macros_cell(const orc_params *p, const double g[Q], double phi, const double grad[3],
                     double lap, double *rho, double *P, double u[3], double *mu) {
    double rho_dif = p->rho_H - p->rho_L;
    *rho = p->rho_L + phi * rho_dif;
    *mu = orc_chem_pot(p, phi, lap);
    double m[3] = {0, 0, 0}, s = 0;
    for (int i = 0; i < Q; ++i) {
        s += g[i];
        m[0] += CX[i] * g[i];
        m[1] += CY[i] * g[i];
        m[2] += CZ[i] * g[i];
    }
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * (*mu * grad[a] + p->Fex[a])) / *rho;
    double ug = u[0] * grad[0] + u[1] * grad[1] + u[2] * grad[2];
    *P = TT * s + 0.5 * TT * rho_dif * ug;
}

/* Force term K_i of Eq. 6 and the pieces of the equilibrium of Eq. 6:
 * E_i = rho Gamma_i + w_i (P/T - rho), g_eq_i = E_i - K_i/2. */
void orc_force_and_eq(const orc_params *p, double rho, double P, const double u[3], double mu,
                      const double grad[3], double K[Q], double E[Q]) {
    double G[Q];
    orc_gamma(u, G);
    double rho_dif = p->rho_H - p->rho_L;
    for (int i = 0; i < Q; ++i) {
        double cmu[3] = {CX[i] - u[0], CY[i] - u[1], CZ[i] - u[2]};
        double cg = cmu[0] * grad[0] + cmu[1] * grad[1] + cmu[2] * grad[2];
        double cF = cmu[0] * p->Fex[0] + cmu[1] * p->Fex[1] + cmu[2] * p->Fex[2];
        K[i] = ((G[i] - WQ[i]) * rho_dif + G[i] * mu / TT) * cg + G[i] * cF / TT;
        E[i] = rho * G[i] + WQ[i] * (P / TT - rho);
    }
}

/* Filtered collision of Eqs. 9-11 (reading R2):
 *   gstar_i = (E_i + K_i/2) + (1 - 1/tau) Phi_i : Pi,
 *   Phi_i = w_i/(2T^2) (c_i c_i - T I),  Pi = sum_l c_l c_l (g_l - g_eq_l).
 * Also returns Pi (row-major 3x3) when Pi_out is not NULL. */
void orc_filtered_collide(const double g[Q], const double K[Q], const double E[Q], double tau,
                          double gstar[Q], double *Pi_out) {
    double Pi[3][3] = {{0}};
    for (int l = 0; l < Q; ++l) {
        double neq = g[l] - (E[l] - 0.5 * K[l]);
        int c[3] = {CX[l], CY[l], CZ[l]};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Pi[a][b] += c[a] * c[b] * neq;
    }
    double trPi = Pi[0][0] + Pi[1][1] + Pi[2][2];
    for (int i = 0; i < Q; ++i) {
        int c[3] = {CX[i], CY[i], CZ[i]};
        double ccPi = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) ccPi += c[a] * c[b] * Pi[a][b];
        double PhiPi = WQ[i] / (2.0 * TT * TT) * (ccPi - TT * trPi);
        gstar[i] = E[i] + 0.5 * K[i] + (1.0 - 1.0 / tau) * PhiPi;
    }
    if (Pi_out)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Pi_out[3 * a + b] = Pi[a][b];
}

/* Wettability ghosts of Sec. II B (Eqs. 12-15) for one wall node:
 * w = n_w rotated by pi - theta about n_w x grad (R9), then for every
 * ghost link i, phi_{s,i} = (1 + tanh((x - x0 + d_i)/(W/2)))/2 with
 * x - x0 = (W/2) artanh(2 phi_smpl - 1) and d_i = w . c_i.
 * links: bit i set when x + c_i is solid (or cut, R23).  Writes out[i] for
 * those. */
void orc_ghost_values(const orc_params *p, double phi_smpl, const double nw[3], double cth,
                      double sth, const double grad[3], uint32_t links, double out[Q]) {
    double gn = grad[0] * nw[0] + grad[1] * nw[1] + grad[2] * nw[2];
    double gt[3] = {grad[0] - gn * nw[0], grad[1] - gn * nw[1], grad[2] - gn * nw[2]};
    double gtn = sqrt(gt[0] * gt[0] + gt[1] * gt[1] + gt[2] * gt[2]);
    double t[3] = {0, 0, 0};
    if (gtn >= 1e-10) {
        t[0] = gt[0] / gtn;
        t[1] = gt[1] / gtn;
        t[2] = gt[2] / gtn;
    }
    double w[3];
    for (int a = 0; a < 3; ++a) w[a] = -cth * nw[a] + sth * t[a];
    double s = 2.0 * phi_smpl - 1.0;
    const double lim = 1.0 - 1e-12;
    if (s > lim) s = lim;
    if (s < -lim) s = -lim;
    double xx0 = 0.5 * p->W * atanh(s); /* Eq. 14 */
    for (int i = 1; i < Q; ++i) {
        if (!(links >> i & 1u)) continue;
        double di = w[0] * CX[i] + w[1] * CY[i] + w[2] * CZ[i];
        out[i] = 0.5 * (1.0 + tanh((xx0 + di) / (0.5 * p->W))); /* Eq. 15 */
    }
}

/* Specular-reflection partner of edge link i at fluid cell x (reading R14):
 * returns the tangential neighbour y and sets *r to the reflected direction,
 * or -1 when the link is not a flat-wall edge link. */
static int64_t specular_partner(const orc_lattice *L, int64_t x, int i, int *r) {
    int c[3] = {CX[i], CY[i], CZ[i]};
    int nz = (c[0] != 0) + (c[1] != 0) + (c[2] != 0);
    if (nz != 2) return -1;
    int a = -1, b = -1;
    for (int k = 0; k < 3; ++k) {
        if (c[k] == 0) continue;
        if (a < 0) a = k; else b = k;
    }
    int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
    ea[a] = c[a];
    eb[b] = c[b];
    int sa = L->solid[shift(L, x, ea[0], ea[1], ea[2])];
    int sb = L->solid[shift(L, x, eb[0], eb[1], eb[2])];
    int wall_axis, tang[3];
    if (sa && !sb) { wall_axis = a; memcpy(tang, eb, sizeof tang); }
    else if (sb && !sa) { wall_axis = b; memcpy(tang, ea, sizeof tang); }
    else return -1;
    int64_t y = shift(L, x, tang[0], tang[1], tang[2]);
    int cr[3] = {c[0], c[1], c[2]};
    cr[wall_axis] = -cr[wall_axis];
    for (int k = 0; k < Q; ++k)
        if (CX[k] == cr[0] && CY[k] == cr[1] && CZ[k] == cr[2]) { *r = k; return y; }
    return -1;
}

/* ----------------------------------------------------- lattice lifecycle */

orc_lattice *orc_create(int nx, int ny, int nz, const uint8_t *solid, const double *wall_normal,
                        const double *theta_deg, const orc_params *p) {
    orc_lattice *L = (orc_lattice *)calloc(1, sizeof *L);
    if (!L) return NULL;
    L->nx = nx; L->ny = ny; L->nz = nz;
    L->N = (int64_t)nx * ny * nz;
    L->p = *p;
    int64_t N = L->N;
    L->solid = (uint8_t *)malloc(N);
    L->nw = (double *)calloc(N * 3, sizeof(double));
    L->cth = (double *)malloc(N * sizeof(double));
    L->sth = (double *)malloc(N * sizeof(double));
    L->h = (double *)calloc(N * Q, sizeof(double));
    L->g = (double *)calloc(N * Q, sizeof(double));
    L->h2 = (double *)calloc(N * Q, sizeof(double));
    L->g2 = (double *)calloc(N * Q, sizeof(double));
    L->phi = (double *)calloc(N, sizeof(double));
    L->ghost = (double *)calloc(N * Q, sizeof(double));
    L->ghost_old = (double *)calloc(N * Q, sizeof(double));
    memcpy(L->solid, solid, N);
    for (int64_t c = 0; c < N; ++c) {
        double th = (theta_deg ? theta_deg[c] : p->theta_deg) * M_PI / 180.0;
        L->cth[c] = cos(th);
        L->sth[c] = sin(th);
        if (!is_wall_node(L, c)) continue;
        if (wall_normal) {
            for (int a = 0; a < 3; ++a) L->nw[3 * c + a] = wall_normal[3 * c + a];
        } else {
            /* Fallback normal from the mask: -sum_i w_i c_i chi_solid(x+c_i). */
            double n[3] = {0, 0, 0};
            for (int i = 1; i < Q; ++i)
                if (L->solid[nbr(L, c, i)]) {
                    n[0] -= WQ[i] * CX[i];
                    n[1] -= WQ[i] * CY[i];
                    n[2] -= WQ[i] * CZ[i];
                }
            double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            if (nn > 0)
                for (int a = 0; a < 3; ++a) L->nw[3 * c + a] = n[a] / nn;
        }
    }
    return L;
}

void orc_destroy(orc_lattice *L) {
    if (!L) return;
    free(L->solid); free(L->frac); free(L->cn); free(L->nw); free(L->cth); free(L->sth);
    free(L->h); free(L->g); free(L->h2); free(L->g2);
    free(L->phi); free(L->ghost); free(L->ghost_old); free(L->bstate);
    free(L);
}

/* Solid volume fractions of the cells (R23), before orc_init_phi: frac[c]
 * in [0, 1) on fluid cells (solid cells count 1 whatever is given).  Wall
 * normals of the wall nodes this adds come from wall_normal, else from the
 * fraction-weighted mask -sum_i w_i c_i s(x + c_i).  Returns 0, or -1 for a
 * fraction out of range. */
int orc_set_solid_fraction(orc_lattice *L, const double *frac, const double *wall_normal) {
    int64_t N = L->N;
    if (N <= 0) return -1;
    for (int64_t c = 0; c < N; ++c)
        if (!L->solid[c] && !(frac[c] >= 0.0 && frac[c] < 1.0)) return -1;
    if (!L->frac) L->frac = (double *)malloc(N * sizeof(double));
    if (!L->cn) L->cn = (int8_t *)calloc((size_t)N, 1);
    for (int64_t c = 0; c < N; ++c) L->frac[c] = L->solid[c] ? 1.0 : frac[c];
    for (int64_t c = 0; c < N; ++c) {
        L->cn[c] = 0;
        if (!is_wall_node(L, c)) continue;
        double *n = L->nw + 3 * c;
        if (wall_normal) {
            for (int a = 0; a < 3; ++a) n[a] = wall_normal[3 * c + a];
        } else {
            n[0] = n[1] = n[2] = 0.0;
            for (int i = 1; i < Q; ++i) {
                double s = sfrac(L, nbr(L, c, i));
                n[0] -= WQ[i] * CX[i] * s;
                n[1] -= WQ[i] * CY[i] * s;
                n[2] -= WQ[i] * CZ[i] * s;
            }
            double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            for (int a = 0; a < 3; ++a) n[a] = nn > 0 ? n[a] / nn : 0.0;
        }
        /* c_n: the axis direction (1..6) with the largest c . n_w */
        double best = 0.0;
        for (int i = 1; i <= 6; ++i) {
            double d = CX[i] * n[0] + CY[i] * n[1] + CZ[i] * n[2];
            if (d > best) { best = d; L->cn[c] = (int8_t)i; }
        }
    }
    return 0;
}

/* Neighbour values for the CD stencil at fluid cell x: phi of fluid
 * neighbours, the wall node's ghost for solid ones (Sec. II B). */
/* Link i of x points into the wall: c_i . n_w(x) < 0 (R23). */
static inline int into_wall(const orc_lattice *L, int64_t x, int i) {
    const double *n = L->nw + 3 * x;
    return CX[i] * n[0] + CY[i] * n[1] + CZ[i] * n[2] < -1e-9;
}

static void stencil_values(const orc_lattice *L, int64_t x, const double *ghost, double val[Q]) {
    val[0] = L->phi[x];
    for (int i = 1; i < Q; ++i) {
        int64_t y = nbr(L, x, i);
        double s = sfrac(L, y);
        if (s >= 1.0)
            val[i] = ghost[x * Q + i];
        else if (s > 0.0 && into_wall(L, x, i)) /* R23: ghost for y's part inside the wall */
            val[i] = s * ghost[x * Q + i] + (1.0 - s) * L->phi[y];
        else
            val[i] = L->phi[y];
    }
}

/* Links of x that carry a ghost: bit i set when x + c_i is solid, or cut
 * with link i pointing into the wall. */
static uint32_t ghost_links(const orc_lattice *L, int64_t x) {
    uint32_t m = 0;
    for (int i = 1; i < Q; ++i) {
        double s = sfrac(L, nbr(L, x, i));
        if (s >= 1.0 || (s > 0.0 && into_wall(L, x, i))) m |= 1u << i;
    }
    return m;
}

/* phi_smpl of wall node x (R6; R23 with a cut cell). */
static double phi_sample(const orc_lattice *L, int64_t x) {
    double sx = L->frac ? L->frac[x] : 0.0;
    if (sx <= 0.0 || L->cn[x] <= 0) return L->phi[x];
    int64_t y = nbr(L, x, L->cn[x]);
    double py = L->solid[y] ? L->phi[x] : L->phi[y];
    return (1.0 - sx) * L->phi[x] + sx * py;
}

/* Equilibrium initialisation (reading R16). */
void orc_init_phi(orc_lattice *L, const double *phi0, double P0) {
    int64_t N = L->N;
    for (int64_t c = 0; c < N; ++c) L->phi[c] = L->solid[c] ? 0.0 : phi0[c];
    for (int64_t c = 0; c < N; ++c) {
        for (int i = 0; i < Q; ++i) L->ghost[c * Q + i] = L->phi[c];
    }
    const orc_params *p = &L->p;
    for (int64_t c = 0; c < N; ++c) {
        double *h = L->h + c * Q, *g = L->g + c * Q;
        if (L->solid[c]) {
            for (int i = 0; i < Q; ++i) h[i] = g[i] = 0.0;
            continue;
        }
        double val[Q], grad[3], lap;
        stencil_values(L, c, L->ghost, val);
        orc_cd_stencil(val, grad, &lap);
        double u[3] = {0, 0, 0};
        orc_h_eq(p, L->phi[c], u, grad, lap, h);
        double rho = p->rho_L + L->phi[c] * (p->rho_H - p->rho_L);
        double mu = orc_chem_pot(p, L->phi[c], lap);
        double K[Q], E[Q];
        orc_force_and_eq(p, rho, P0, u, mu, grad, K, E);
        for (int i = 0; i < Q; ++i) g[i] = E[i] - 0.5 * K[i];
    }
    L->step = 0;
}

/* --------------------------------------------------- open boundaries (R22) */

/* Given boundary value k (P, ux, uy, uz, phi) of side s at step t: linear
 * from bc_from at step bc_t0 to bc_val at step bc_t0 + bc_ramp. */
static double bc_value(const orc_lattice *L, int s, int k, int64_t t) {
    if (L->bc_ramp <= 0 || t >= L->bc_t0 + L->bc_ramp) return L->bc_val[s][k];
    double f = t <= L->bc_t0 ? 0.0 : (double)(t - L->bc_t0) / (double)L->bc_ramp;
    return L->bc_from[s][k] + f * (L->bc_val[s][k] - L->bc_from[s][k]);
}

static inline int bc_side(const orc_lattice *L, int64_t c) {
    if (!L->bc_type[0] || L->solid[c]) return -1;
    int64_t x = c % L->nx;
    return x == 0 ? 0 : (x == L->nx - 1 ? 1 : -1);
}

/* Boundary states from the current (post-stream) populations, then phi of
 * the boundary cells := phi_b.  Needs phi of the interior cells. */
static void boundary_states(orc_lattice *L) {
    const orc_params *p = &L->p;
    int64_t plane = (int64_t)L->ny * L->nz;
    for (int side = 0; side < 2 && L->bc_type[0]; ++side) {
        int xb = side ? L->nx - 1 : 0, xa = side ? L->nx - 2 : 1;
        for (int64_t j = 0; j < plane; ++j) {
            int64_t yz = j * L->nx;                 /* y + ny z, times nx */
            int64_t cb = xb + yz, ca = xa + yz;
            double *st = L->bstate + (side * plane + j) * 5;
            double v[5];
            for (int k = 0; k < 5; ++k) v[k] = bc_value(L, side, k, L->step);
            double phia = 0, Pa = 0, ua[3] = {0, 0, 0};
            if (!L->solid[ca]) {
                const double *g = L->g + ca * Q;
                double s0 = 0, m[3] = {0, 0, 0};
                for (int i = 0; i < Q; ++i) {
                    s0 += g[i];
                    m[0] += CX[i] * g[i]; m[1] += CY[i] * g[i]; m[2] += CZ[i] * g[i];
                }
                phia = L->phi[ca];
                double rho = p->rho_L + phia * (p->rho_H - p->rho_L);
                for (int a = 0; a < 3; ++a) ua[a] = (m[a] + 0.5 * p->Fex[a]) / rho;
                Pa = TT * s0;
            }
            if (L->bc_type[side] == 1) {      /* pressure */
                st[0] = phia; st[1] = v[0]; st[2] = ua[0]; st[3] = ua[1]; st[4] = ua[2];
            } else {                          /* velocity */
                st[0] = v[4]; st[1] = Pa; st[2] = v[1]; st[3] = v[2]; st[4] = v[3];
            }
            if (!L->solid[cb]) L->phi[cb] = st[0];
        }
    }
}

/* Post-collision populations of a boundary cell: equilibria at its state. */
static void boundary_equilibria(const orc_lattice *L, int64_t c, int side, double hs[Q],
                                double gs[Q]) {
    const orc_params *p = &L->p;
    int64_t j = c / L->nx;
    const double *st = L->bstate + (side * (int64_t)L->ny * L->nz + j) * 5;
    double u[3] = {st[2], st[3], st[4]}, G[Q];
    orc_gamma(u, G);
    double rho = p->rho_L + st[0] * (p->rho_H - p->rho_L);
    for (int i = 0; i < Q; ++i) {
        hs[i] = st[0] * G[i];
        gs[i] = WQ[i] * st[1] / TT + rho * (G[i] - WQ[i]);
    }
}

/* phi = sum_i h_i on fluid cells (Sec. II A, after Eq. 3). */
static void compute_phi(orc_lattice *L) {
    int64_t N = L->N;
#pragma omp parallel for num_threads(L->p.nthreads) schedule(static)
    for (int64_t c = 0; c < N; ++c) {
        if (L->solid[c]) { L->phi[c] = 0.0; continue; }
        double s = 0;
        for (int i = 0; i < Q; ++i) s += L->h[c * Q + i];
        L->phi[c] = s;
    }
}

/* Ghost update at every wall node (Sec. II B with the blend of Sec. III A):
 * grad phi with the previous ghosts (R11), new ghosts, then the blend. */
static void update_ghosts(orc_lattice *L, double *ghost_out) {
    int64_t N = L->N;
    memcpy(L->ghost_old, L->ghost, N * Q * sizeof(double));
    const orc_params *p = &L->p;
#pragma omp parallel for num_threads(L->p.nthreads) schedule(static)
    for (int64_t c = 0; c < N; ++c) {
        if (L->solid[c] || bc_side(L, c) >= 0) continue;  /* R22: no ghost update */
        uint32_t m = ghost_links(L, c);
        if (!m) continue;
        double val[Q], grad[3], lap, fresh[Q];
        stencil_values(L, c, L->ghost_old, val);
        orc_cd_stencil(val, grad, &lap);
        orc_ghost_values(p, phi_sample(L, c), L->nw + 3 * c, L->cth[c], L->sth[c], grad, m,
                         fresh);
        for (int i = 1; i < Q; ++i)
            if (m >> i & 1u)
                ghost_out[c * Q + i] = p->blend * L->ghost_old[c * Q + i] + (1.0 - p->blend) * fresh[i];
    }
}

/* Macroscopic fields of the current state (phi, rho, P, u), computed the
 * way the next step would: ghosts are updated into a scratch copy. */
void orc_macros(orc_lattice *L, double *phi, double *rho, double *P, double *ux, double *uy,
                double *uz) {
    int64_t N = L->N;
    compute_phi(L);
    double *gs = (double *)malloc(N * Q * sizeof(double));
    boundary_states(L);
    memcpy(gs, L->ghost, N * Q * sizeof(double));
    update_ghosts(L, gs);
    const orc_params *p = &L->p;
#pragma omp parallel for num_threads(L->p.nthreads) schedule(static)
    for (int64_t c = 0; c < N; ++c) {
        if (L->solid[c]) {
            phi[c] = rho[c] = P[c] = ux[c] = uy[c] = uz[c] = 0.0;
            continue;
        }
        const int side = bc_side(L, c);
        if (side >= 0) {  /* R22: the boundary state */
            const double *st = L->bstate + (side * (int64_t)L->ny * L->nz + c / L->nx) * 5;
            phi[c] = st[0];
            rho[c] = p->rho_L + st[0] * (p->rho_H - p->rho_L);
            P[c] = st[1];
            ux[c] = st[2]; uy[c] = st[3]; uz[c] = st[4];
            continue;
        }
        double val[Q], grad[3], lap, r, pr, u[3], mu;
        stencil_values(L, c, gs, val);
        orc_cd_stencil(val, grad, &lap);
        orc_macros_cell(p, L->g + c * Q, L->phi[c], grad, lap, &r, &pr, u, &mu);
        phi[c] = L->phi[c];
        rho[c] = r;
        P[c] = pr;
        ux[c] = u[0]; uy[c] = u[1]; uz[c] = u[2];
    }
    free(gs);
}

/* One time step n -> n+1 in the order of reading R3. */
static void one_step(orc_lattice *L) {
    const orc_params *p = &L->p;
    int64_t N = L->N;
    compute_phi(L);                 /* step 1 */
    boundary_states(L);             /* R22 */
    double *gnew = (double *)malloc(N * Q * sizeof(double));
    memcpy(gnew, L->ghost, N * Q * sizeof(double));
    update_ghosts(L, gnew);         /* step 2 */
    memcpy(L->ghost, gnew, N * Q * sizeof(double));
    free(gnew);
    memset(L->h2, 0, N * Q * sizeof(double));
    memset(L->g2, 0, N * Q * sizeof(double));
    double tau_phi = p->M / TT + 0.5; /* Eq. 1 */
#pragma omp parallel for num_threads(L->p.nthreads) schedule(static)
    for (int64_t c = 0; c < N; ++c) {
        if (L->solid[c]) continue;
        const int side = bc_side(L, c);
        if (side >= 0) {                                 /* R22 */
            double hs[Q], gs[Q];
            boundary_equilibria(L, c, side, hs, gs);
            for (int i = 0; i < Q; ++i) {
                int64_t y = nbr(L, c, i);
                if (!L->solid[y]) {
                    L->h2[y * Q + i] = hs[i];
                    L->g2[y * Q + i] = gs[i];
                } else {
                    L->h2[c * Q + OPP[i]] = hs[i];
                    L->g2[c * Q + OPP[i]] = gs[i];
                }
            }
            continue;
        }
        const double *h = L->h + c * Q, *g = L->g + c * Q;
        double val[Q], grad[3], lap;                     /* step 3 */
        stencil_values(L, c, L->ghost, val);
        orc_cd_stencil(val, grad, &lap);
        double phi = L->phi[c], rho, P, u[3], mu;        /* step 4 */
        orc_macros_cell(p, g, phi, grad, lap, &rho, &P, u, &mu);
        double tau = orc_tau_mix(p, phi);
        double heq[Q], hs[Q];                            /* step 5: Eq. 1 */
        orc_h_eq(p, phi, u, grad, lap, heq);
        for (int i = 0; i < Q; ++i) hs[i] = h[i] - (h[i] - heq[i]) / tau_phi;
        double K[Q], E[Q], gs[Q];                        /* step 6: Eqs. 5-11 */
        orc_force_and_eq(p, rho, P, u, mu, grad, K, E);
        orc_filtered_collide(g, K, E, tau, gs, NULL);
        /* step 7: push streaming.  Each target slot has exactly one
         * writer, so the parallel loop is race free. */
        for (int i = 0; i < Q; ++i) {
            int64_t y = nbr(L, c, i);
            if (!L->solid[y]) {
                L->h2[y * Q + i] = hs[i];
                L->g2[y * Q + i] = gs[i];
                continue;
            }
            L->h2[c * Q + OPP[i]] = hs[i];
            int r;
            int64_t yt = p->free_slip ? specular_partner(L, c, i, &r) : -1;
            if (yt >= 0 && phi >= p->band_lo && phi <= p->band_hi && L->phi[yt] >= p->band_lo &&
                L->phi[yt] <= p->band_hi)
                L->g2[yt * Q + r] = gs[i];
            else
                L->g2[c * Q + OPP[i]] = gs[i];
        }
    }
    double *t;
    t = L->h; L->h = L->h2; L->h2 = t;
    t = L->g; L->g = L->g2; L->g2 = t;
    L->step++;
}

void orc_step(orc_lattice *L, int64_t nsteps) {
    for (int64_t s = 0; s < nsteps; ++s) one_step(L);
}

/* ------------------------------------------------------ state accessors */

int64_t orc_get_step(const orc_lattice *L) { return L->step; }
void orc_get_h(const orc_lattice *L, double *out) { memcpy(out, L->h, L->N * Q * sizeof(double)); }
void orc_get_g(const orc_lattice *L, double *out) { memcpy(out, L->g, L->N * Q * sizeof(double)); }
void orc_set_h(orc_lattice *L, const double *in) { memcpy(L->h, in, L->N * Q * sizeof(double)); }
void orc_set_g(orc_lattice *L, const double *in) { memcpy(L->g, in, L->N * Q * sizeof(double)); }
void orc_get_ghost(const orc_lattice *L, double *out) { memcpy(out, L->ghost, L->N * Q * sizeof(double)); }
void orc_set_ghost(orc_lattice *L, const double *in) { memcpy(L->ghost, in, L->N * Q * sizeof(double)); }
void orc_set_phi_field(orc_lattice *L, const double *in) { memcpy(L->phi, in, L->N * sizeof(double)); }
void orc_get_normals(const orc_lattice *L, double *out) { memcpy(out, L->nw, L->N * 3 * sizeof(double)); }
/* Ghost update on the stored phi field (no step): used by the wetting pin. */
void orc_update_ghosts_only(orc_lattice *L) {
    double *gnew = (double *)malloc(L->N * Q * sizeof(double));
    memcpy(gnew, L->ghost, L->N * Q * sizeof(double));
    update_ghosts(L, gnew);
    memcpy(L->ghost, gnew, L->N * Q * sizeof(double));
    free(gnew);
}
void orc_set_nthreads(orc_lattice *L, int n) { L->p.nthreads = n > 0 ? n : 1; }

/* Open x boundaries (R22): types 0 (both: periodic), 1 pressure, 2 velocity;
 * values P, ux, uy, uz, phi per side.  Returns 0, or -1 for a bad request. */
int orc_set_x_boundaries(orc_lattice *L, int type_lo, const double *val_lo, int type_hi,
                         const double *val_hi, int64_t ramp) {
    if ((type_lo == 0) != (type_hi == 0) || type_lo < 0 || type_lo > 2 || type_hi < 0 ||
        type_hi > 2 || ramp < 0 || (type_lo && (L->nx < 3 || !val_lo || !val_hi)))
        return -1;
    /* ramp start: the values in effect now for an unchanged type, else the
     * rest state (P = 0, u = 0, phi at its target) */
    const int type[2] = {type_lo, type_hi};
    const double *val[2] = {val_lo, val_hi};
    double from[2][5];
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < 5; ++k)
            from[s][k] = (L->bc_type[s] && L->bc_type[s] == type[s]) ? bc_value(L, s, k, L->step)
                         : (k < 4 ? 0.0 : (type[s] ? val[s][4] : 0.0));
    for (int s = 0; s < 2; ++s) {
        L->bc_type[s] = type[s];
        for (int k = 0; k < 5; ++k) {
            L->bc_val[s][k] = type[s] ? val[s][k] : 0.0;
            L->bc_from[s][k] = from[s][k];
        }
    }
    L->bc_t0 = L->step;
    L->bc_ramp = ramp;
    if (type_lo && !L->bstate)
        L->bstate = (double *)calloc((size_t)2 * L->ny * L->nz * 5, sizeof(double));
    return 0;
}
void orc_set_force(orc_lattice *L, const double F[3]) {
    for (int a = 0; a < 3; ++a) L->p.Fex[a] = F[a];
}
void orc_lattice_tables(int *cx, int *cy, int *cz, double *w, int *opp) {
    for (int i = 0; i < Q; ++i) {
        cx[i] = CX[i]; cy[i] = CY[i]; cz[i] = CZ[i]; w[i] = WQ[i]; opp[i] = OPP[i];
    }
}
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

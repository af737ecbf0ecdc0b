/*
 * Plain FP64 CPU oracle of the phase-field WMRT lattice Boltzmann time step
 * (conservative Allen-Cahn populations g + pressure-based hydrodynamic
 * populations f, D2Q9 and D3Q19).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it; the product library never links, calls or imports it, and the
 * two share no code, headers or tables.
 *
 * Every formula is written in the paper's order and notation (lattice units,
 * dx = dt = c = 1, c_s^2 = 1/3, phi_L = 0, phi_H = 1, phi_0 = 1/2):
 *   Sec. 3.1  eq:chemical_potential, eq:beta_kappa_relation,
 *             eq:surface_tension_force
 *   Sec. 3.2  eq:lbe_standard .. eq:density_gradient_phase_field (f-LBE),
 *             eq:lbe_interface .. eq:laplacian_phi (g-LBE and stencils)
 *   App. A    eq:A1 (D2Q9 M), eq:A2 (D3Q19 weighted M), eq:23 (S-hat)
 *   App. B    periodic (eq:streaming_f/g, eq:periodic_*), halfway bounce-back
 *             (eq:no_slip_f/g), velocity and phase inlet
 *             (eq:velocity_boundary_*, eq:mass_conservation ..
 *             eq:unknown_distribution_tangential), convective outlet
 *             (eq:implicit_convective, eq:convective_f/g)
 *   Sec. 6.1  eq:gravity_force (body force with a reference density)
 *
 * Readings where the paper is silent, garbled or inconsistent (each is marked
 * "Reading" at the place it is used):
 *   R1  eq:chemical_potential prints +4 beta phi(1-phi)(phi-1/2); that sign
 *       makes the tanh profile of eq:kernel_function a non-equilibrium.  The
 *       oracle uses 4 beta (phi-phi_L)(phi-phi_H)(phi-phi_0) - kappa lap(phi).
 *   R2  F_mu needs f^eq(u) and u needs F_mu.  The oracle evaluates F_mu with
 *       f^eq(p*, u0), u0 = sum f e + (F_s + F_p + F_b)/(2 rho), then forms the
 *       final u; the state is the populations alone.
 *   R3  eq:relaxation_time (tau linear in phi) and eq:dynamic_viscosity (mu
 *       linear in phi) cannot both hold.  visc_model = 0 (default) makes mu
 *       linear, tau = mu(phi) / (rho(phi) c_s^2) with mu_X = rho_X tau_X c_s^2;
 *       visc_model = 1 makes tau linear.  (With tau linear, the 128^2 drop at
 *       density ratio 1000, viscosity ratio 100, tau_H = 0.8 diverges within
 *       100 steps; with mu linear it is stable.)
 *   R4  phi is clamped to [0,1] inside rho, tau (and mu) only.
 *   R5  D2Q9 S-hat is not printed; rows p_xx, p_xy of eq:A1 relax at s_nu,
 *       all other rows at 1, as eq:23 does for D3Q19.
 *   R6  ghost phi: periodic -> wrapped value; wall and outlet -> value of the
 *       adjacent fluid node (zero normal gradient); inlet -> phi_in.
 *   R7  n = grad(phi)/|grad(phi)| is taken as 0 where |grad(phi)| < 1e-12.
 *   R8  inlet: derivatives of phi are not evaluated at inlet nodes (the
 *       paper treats the inlet as single phase and skips the derivatives of
 *       the macroscopic variables there): grad phi = lap phi = 0, so the
 *       interfacial forces F_s, F_p, F_mu and F^phi vanish at inlet nodes;
 *       the velocity rule is applied to f' = f + F/2 with the force that
 *       remains, the body force F_b = (rho(phi_in) - rho_ref) g, so that
 *       sum f' e = u_in (eq:velocity_boundary_u) and the velocity of the next
 *       macroscopic update is u_in;
 *       p* cancels from eq:velocity_boundary_distribution; the tangential
 *       excess momentum is shared by the 2 unknown populations that carry each
 *       tangential component (factor 1/2, which makes
 *       eq:velocity_boundary_u hold exactly); the phase-field excess theta is
 *       shared by the N unknown populations that have a tangential component
 *       (N = 2 in D2Q9, 4 in D3Q19), which makes eq:mass_conservation hold
 *       exactly; nozzle profile phi_in = 1/2 + 1/2 tanh(2(R - r)/W), plug
 *       velocity u_j inside r < R, zero outside.
 *   R9  outlet: U_local = sum_a f_a e_a . n at the (N-1) layer after
 *       streaming (bare first moment of the distribution), lambda clamped to
 *       [0,1]; the blend is applied to every population of both sets.
 *   The inlet is only allowed on the low face and the outlet on the high face
 *   of the last axis (y in 2D, z in 3D).
 *
 * Layout inside the oracle: node-major, pop[node * Q + a], node =
 * (z * ny + y) * nx + x.  The exported population arrays are population-major
 * [a][z][y][x].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 19

enum { ORC_D2Q9 = 0, ORC_D3Q19 = 1 };
enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET = 2, BC_OUTFLOW = 3, BC_FREESLIP = 4 };

typedef struct {
    int32_t lattice, nx, ny, nz;
    int32_t bc[6];           /* faces -x,+x,-y,+y,-z,+z */
    int32_t visc_model;      /* 0: mu linear in phi, 1: tau linear in phi */
    int32_t outlet_scheme;   /* outlet speed U of eq:velocity_options: 0 local, 1 max, 2 average */
    double rho_L, rho_H, tau_L, tau_H;
    double mu_ratio;         /* mu_H / mu_L; when > 0 it sets tau_L (Reading R3) */
    double sigma, W, mobility;
    double force[3];         /* body-force acceleration g */
    double rho_ref;          /* F_b = (rho - rho_ref) g */
    double inlet_u;          /* plug speed along the inward normal */
    double inlet_center[2];  /* nozzle centre in the inlet plane */
    double inlet_radius;     /* nozzle radius (2D: half width) */
} orc_params;

typedef struct {
    orc_params p;
    int Q, D, L;             /* L: last axis (inlet/outlet axis) */
    int n[3];
    int64_t N;
    int e[QMAX][3];
    double w[QMAX];
    int opp[QMAX];
    double M[QMAX][QMAX];
    double Minv[QMAX][QMAX];
    int shear[QMAX];         /* 1 for rows relaxed at s_nu */
    double *fA, *gA, *fB, *gB, *fs, *gs, *phi;
} orc_ctx;

static const double CS2 = 1.0 / 3.0;

/* ---------------------------------------------------------------- lattices */

/* eq:A1, App. A: D2Q9 transformation matrix, printed row by row. */
static const int M_D2Q9[9][9] = {
    { 1,  1,  1,  1,  1,  1,  1,  1,  1},
    {-4, -1, -1, -1, -1,  2,  2,  2,  2},
    { 4, -2, -2, -2, -2,  1,  1,  1,  1},
    { 0,  1,  0, -1,  0,  1, -1, -1,  1},
    { 0, -2,  0,  2,  0,  1, -1, -1,  1},
    { 0,  0,  1,  0, -1,  1,  1, -1, -1},
    { 0,  0, -2,  0,  2,  1,  1, -1, -1},
    { 0,  1, -1,  1, -1,  0,  0,  0,  0},
    { 0,  0,  0,  0,  0,  1, -1,  1, -1},
};

/* eq:A2, App. A: D3Q19 weighted transformation matrix, printed row by row. */
static const int M_D3Q19[19][19] = {
    { 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    { 0, 1,-1, 0, 0, 0, 0, 1,-1, 1,-1, 1,-1, 1,-1, 0, 0, 0, 0},
    { 0, 0, 0, 1,-1, 0, 0, 1,-1,-1, 1, 0, 0, 0, 0, 1,-1, 1,-1},
    { 0, 0, 0, 0, 0, 1,-1, 0, 0, 0, 0, 1,-1,-1, 1, 1,-1,-1, 1},
    { 0, 0, 0, 0, 0, 0, 0, 1, 1,-1,-1, 0, 0, 0, 0, 0, 0, 0, 0},
    { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1,-1,-1},
    { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1,-1,-1, 0, 0, 0, 0},
    { 0, 2, 2,-1,-1,-1,-1, 1, 1, 1, 1, 1, 1, 1, 1,-2,-2,-2,-2},
    { 0, 0, 0, 1, 1,-1,-1, 1, 1, 1, 1,-1,-1,-1,-1, 0, 0, 0, 0},
    {-1, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    { 0,-2, 2, 0, 0, 0, 0, 1,-1, 1,-1, 1,-1, 1,-1, 0, 0, 0, 0},
    { 0, 0, 0,-2, 2, 0, 0, 1,-1,-1, 1, 0, 0, 0, 0, 1,-1, 1,-1},
    { 0, 0, 0, 0, 0,-2, 2, 0, 0, 0, 0, 1,-1,-1, 1, 1,-1,-1, 1},
    { 0, 0, 0, 0, 0, 0, 0, 1,-1, 1,-1,-1, 1,-1, 1, 0, 0, 0, 0},
    { 0, 0, 0, 0, 0, 0, 0,-1, 1, 1,-1, 0, 0, 0, 0, 1,-1, 1,-1},
    { 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1,-1,-1, 1,-1, 1, 1,-1},
    { 1,-2,-2,-2,-2,-2,-2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    { 0,-2,-2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,-2,-2,-2,-2},
    { 0, 0, 0,-1,-1, 1, 1, 1, 1, 1, 1,-1,-1,-1,-1, 0, 0, 0, 0},
};

/* Velocity sets: the momentum rows of the printed matrices fix the ordering
 * (eq:A1 rows 4 and 6; eq:A2 rows 2-4).  Weights: eq:weights for D3Q19; the
 * paper prints none for D2Q9, so the standard 4/9, 1/9, 1/36 are used. */
static void fill_lattice(orc_ctx* c, int lattice)
{
    memset(c->e, 0, sizeof c->e);
    memset(c->shear, 0, sizeof c->shear);
    if (lattice == ORC_D2Q9) {
        c->Q = 9; c->D = 2;
        for (int a = 0; a < 9; ++a) {
            c->e[a][0] = M_D2Q9[3][a];
            c->e[a][1] = M_D2Q9[5][a];
            int e2 = c->e[a][0] * c->e[a][0] + c->e[a][1] * c->e[a][1];
            c->w[a] = e2 == 0 ? 4.0 / 9.0 : (e2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
            for (int k = 0; k < 9; ++k) c->M[k][a] = M_D2Q9[k][a];
        }
        c->shear[7] = c->shear[8] = 1;                 /* Reading R5 */
    } else {
        c->Q = 19; c->D = 3;
        for (int a = 0; a < 19; ++a) {
            for (int d = 0; d < 3; ++d) c->e[a][d] = M_D3Q19[1 + d][a];
            int e2 = c->e[a][0] * c->e[a][0] + c->e[a][1] * c->e[a][1] + c->e[a][2] * c->e[a][2];
            c->w[a] = e2 == 0 ? 12.0 / 36.0 : (e2 == 1 ? 2.0 / 36.0 : 1.0 / 36.0);
            for (int k = 0; k < 19; ++k) c->M[k][a] = M_D3Q19[k][a];
        }
        for (int k = 4; k <= 8; ++k) c->shear[k] = 1;  /* eq:23 */
    }
    for (int a = 0; a < c->Q; ++a)
        for (int b = 0; b < c->Q; ++b)
            if (c->e[b][0] == -c->e[a][0] && c->e[b][1] == -c->e[a][1] && c->e[b][2] == -c->e[a][2])
                c->opp[a] = b;
}

/* Inverse of M by Gauss-Jordan elimination with partial pivoting (textbook
 * routine; no use is made of the orthogonality of M). */
static int invert(int Q, double A[QMAX][QMAX], double Ainv[QMAX][QMAX])
{
    double a[QMAX][2 * QMAX];
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < 2 * Q; ++j)
            a[i][j] = j < Q ? A[i][j] : (j - Q == i ? 1.0 : 0.0);
    for (int col = 0; col < Q; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (fabs(a[piv][col]) < 1e-14) return -1;
        if (piv != col)
            for (int j = 0; j < 2 * Q; ++j) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
        double d = a[col][col];
        for (int j = 0; j < 2 * Q; ++j) a[col][j] /= d;
        for (int r = 0; r < Q; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m != 0.0)
                for (int j = 0; j < 2 * Q; ++j) a[r][j] -= m * a[col][j];
        }
    }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) Ainv[i][j] = a[i][Q + j];
    return 0;
}

/* eq:dimensionless_distribution */
static double Gamma(const orc_ctx* c, int a, const double u[3])
{
    double eu = 0.0, uu = 0.0;
    for (int d = 0; d < 3; ++d) { eu += c->e[a][d] * u[d]; uu += u[d] * u[d]; }
    return c->w[a] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* (M^-1 S M) x, eq:mrt_collision, evaluated as M^-1 (S (M x)). */
static void apply_MSM(const orc_ctx* c, double s_nu, const double* x, double* y)
{
    int Q = c->Q;
    double m[QMAX];
    for (int k = 0; k < Q; ++k) {
        double acc = 0.0;
        for (int a = 0; a < Q; ++a) acc += c->M[k][a] * x[a];
        m[k] = (c->shear[k] ? s_nu : 1.0) * acc;
    }
    for (int b = 0; b < Q; ++b) {
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) acc += c->Minv[b][k] * m[k];
        y[b] = acc;
    }
}

/* ------------------------------------------------------- one node, one step */

/* Macroscopic update and collision of one node.
 * f, g: the node's post-stream populations; phin[a] = phi(x + e_a) (phin[0] =
 * phi(x)); inlet_node: the node lies on an inlet face.  Writes the post-collision populations fs, gs (either may be NULL),
 * out = {phi, u_x, u_y, u_z, p} and terms = {phi, dphi/dx, dphi/dy, dphi/dz,
 * lap phi, rho, tau, mu_phi, p*, F_x, F_y, F_z, u_x, u_y, u_z} (may be NULL). */
static void node_update(const orc_ctx* c, const double* f, const double* g, const double* phin,
                        int inlet_node, double* fs, double* gs, double* out, double* terms)
{
    const orc_params* P = &c->p;
    int Q = c->Q;

    /* eq:phase_field_variable */
    double phi = 0.0;
    for (int a = 0; a < Q; ++a) phi += g[a];

    /* eq:gradient_phi, eq:laplacian_phi (not evaluated at inlet nodes, R8) */
    double gphi[3] = {0, 0, 0}, lap = 0.0;
    if (!inlet_node)
        for (int a = 0; a < Q; ++a) {
            for (int d = 0; d < 3; ++d) gphi[d] += c->e[a][d] * c->w[a] * phin[a] / CS2;
            lap += 2.0 * c->w[a] * (phin[a] - phin[0]) / CS2;
        }

    /* Reading R4, eq:density_interpolation, eq:relaxation_time (R3) */
    double ph = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
    double rho = P->rho_L + ph * (P->rho_H - P->rho_L);
    double tau;
    if (P->visc_model == 1) {
        tau = P->tau_L + ph * (P->tau_H - P->tau_L);
    } else {
        double muL = P->rho_L * P->tau_L * CS2, muH = P->rho_H * P->tau_H * CS2;
        double mu = muL + ph * (muH - muL);           /* eq:dynamic_viscosity */
        tau = mu / (rho * CS2);
    }
    double nu = tau * CS2;                            /* eq:kinematic_viscosity */
    double s_nu = 1.0 / (tau + 0.5);                  /* eq:bgk_collision rate */

    /* eq:beta_kappa_relation, eq:chemical_potential (Reading R1),
     * eq:surface_tension_force */
    double beta = 12.0 * P->sigma / P->W, kappa = 3.0 * P->sigma * P->W / 2.0;
    double mu_phi = 4.0 * beta * (phi - 0.0) * (phi - 1.0) * (phi - 0.5) - kappa * lap;
    double Fs[3], Fp[3], Fb[3], gr[3];

    /* eq:normalized_pressure */
    double pstar = 0.0, j[3] = {0, 0, 0};
    for (int a = 0; a < Q; ++a) {
        pstar += f[a];
        for (int d = 0; d < 3; ++d) j[d] += f[a] * c->e[a][d];
    }
    for (int d = 0; d < 3; ++d) {
        Fs[d] = mu_phi * gphi[d];
        gr[d] = (P->rho_H - P->rho_L) * gphi[d];      /* eq:density_gradient_phase_field */
        Fp[d] = -pstar * CS2 * gr[d];                 /* eq:pressure_force */
        Fb[d] = (rho - P->rho_ref) * P->force[d];     /* eq:gravity_force */
    }

    /* Reading R2: predictor velocity, then eq:viscous_force_wmrt */
    double u0[3], feq[QMAX], dneq[QMAX], cd[QMAX];
    for (int d = 0; d < 3; ++d) u0[d] = j[d] + (Fs[d] + Fp[d] + Fb[d]) / (2.0 * rho);
    for (int a = 0; a < Q; ++a) {
        feq[a] = pstar * c->w[a] + (Gamma(c, a, u0) - c->w[a]);   /* eq:equilibrium */
        dneq[a] = f[a] - feq[a];
    }
    apply_MSM(c, s_nu, dneq, cd);
    double Fmu[3];
    for (int i = 0; i < 3; ++i) {
        double acc = 0.0;
        for (int jj = 0; jj < 3; ++jj) {
            double Pi = 0.0;
            for (int b = 0; b < Q; ++b) Pi += c->e[b][i] * c->e[b][jj] * cd[b];
            acc += Pi * gr[jj];
        }
        Fmu[i] = -nu / CS2 * acc;
    }

    /* eq:total_force, eq:velocity_update */
    double F[3], u[3];
    for (int d = 0; d < 3; ++d) {
        F[d] = Fs[d] + Fb[d] + Fp[d] + Fmu[d];
        u[d] = j[d] + F[d] / (2.0 * rho);
    }

    if (gs) {
        /* eq:forcing_term with Reading R7, eq:equilibrium_function,
         * eq:equilibrium_with_force, eq:mobility_relation, eq:lbe_interface */
        double gn = sqrt(gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2]);
        double nrm[3] = {0, 0, 0};
        if (gn >= 1e-12)
            for (int d = 0; d < 3; ++d) nrm[d] = gphi[d] / gn;
        double tau_phi = P->mobility / CS2;
        for (int a = 0; a < Q; ++a) {
            double en = 0.0;
            for (int d = 0; d < 3; ++d) en += c->e[a][d] * nrm[d];
            double Fphi = (1.0 - 4.0 * (phi - 0.5) * (phi - 0.5)) / P->W * c->w[a] * en;
            double geq = phi * Gamma(c, a, u);
            double gbar = geq - 0.5 * Fphi;
            gs[a] = g[a] - (g[a] - gbar) / (tau_phi + 0.5) + Fphi;
        }
    }
    if (fs) {
        /* eq:force_term, eq:equilibrium, eq:equilibrium_modified,
         * eq:mrt_collision, eq:lbe_standard */
        double Fa[QMAX], delta[QMAX], cdel[QMAX];
        for (int a = 0; a < Q; ++a) {
            double eF = 0.0;
            for (int d = 0; d < 3; ++d) eF += c->e[a][d] * F[d];
            Fa[a] = c->w[a] * eF / (rho * CS2);
            double fe = pstar * c->w[a] + (Gamma(c, a, u) - c->w[a]);
            double fbar = fe - 0.5 * Fa[a];
            delta[a] = f[a] - fbar;
        }
        apply_MSM(c, s_nu, delta, cdel);
        for (int a = 0; a < Q; ++a) fs[a] = f[a] - cdel[a] + Fa[a];
    }
    if (terms) {
        terms[0] = phi;
        terms[1] = gphi[0]; terms[2] = gphi[1]; terms[3] = gphi[2];
        terms[4] = lap; terms[5] = rho; terms[6] = tau; terms[7] = mu_phi; terms[8] = pstar;
        terms[9] = F[0]; terms[10] = F[1]; terms[11] = F[2];
        terms[12] = u[0]; terms[13] = u[1]; terms[14] = u[2];
    }
    if (out) {
        out[0] = phi;
        out[1] = u[0]; out[2] = u[1]; out[3] = u[2];
        out[4] = pstar * rho * CS2;                   /* p* = p / (rho c_s^2) */
    }
}

/* ------------------------------------------------------------ grid helpers */

static inline int64_t nid(const orc_ctx* c, int x, int y, int z)
{
    return ((int64_t)z * c->n[1] + y) * c->n[0] + x;
}

/* Nozzle profile of the inlet plane (Reading R8). */
static void inlet_profile(const orc_ctx* c, int t0, int t1, double* phi_in, double* un)
{
    double r;
    if (c->D == 2) r = fabs((double)t0 - c->p.inlet_center[0]);
    else {
        double dx = (double)t0 - c->p.inlet_center[0], dy = (double)t1 - c->p.inlet_center[1];
        r = sqrt(dx * dx + dy * dy);
    }
    *phi_in = 0.5 + 0.5 * tanh(2.0 * (c->p.inlet_radius - r) / c->p.W);
    *un = r < c->p.inlet_radius ? c->p.inlet_u : 0.0;
}

/* phi at the neighbour position v = x + e_a, with ghost values (Reading R6). */
static double phi_at(const orc_ctx* c, const double* phi, const int v[3])
{
    int m[3];
    int inlet = 0;
    for (int d = 0; d < 3; ++d) {
        m[d] = v[d];
        if (v[d] >= 0 && v[d] < c->n[d]) continue;
        int face = 2 * d + (v[d] < 0 ? 0 : 1);
        int bc = c->p.bc[face];
        if (bc == BC_PERIODIC) m[d] = (v[d] + c->n[d]) % c->n[d];
        else {
            m[d] = v[d] < 0 ? 0 : c->n[d] - 1;
            if (bc == BC_INLET) inlet = 1;
        }
    }
    if (inlet) {
        double pin, un;
        inlet_profile(c, m[0], m[1], &pin, &un);
        return pin;
    }
    return phi[nid(c, m[0], m[1], m[2])];
}

/* The node lies on the inlet face (first layer of the last axis). */
static int is_inlet_node(const orc_ctx* c, int x, int y, int z)
{
    int v[3] = {x, y, z};
    return c->p.bc[2 * c->L] == BC_INLET && v[c->L] == 0;
}

/* Fill phin[a] = phi(x + e_a) for node (x,y,z). */
static void gather_phi(const orc_ctx* c, const double* phi, int x, int y, int z, double* phin)
{
    for (int a = 0; a < c->Q; ++a) {
        int v[3] = {x + c->e[a][0], y + c->e[a][1], z + c->e[a][2]};
        phin[a] = phi_at(c, phi, v);
    }
}

/* Classify the pull source of population a at node (x,y,z): returns 0 with
 * the source node and the source direction *asrc (a, or its mirror image
 * after a free-slip reflection), 1 for a wall link (bounce-back), 2 for a link
 * through an open face (unknown, fixed by the inlet/outlet rule).  Free slip
 * (eq:free_slip_f/g, App. B): a population that crossed slip faces was
 * reflected specularly there: it left the node x - e_a with the coordinates
 * of the crossed axes reset to those of x, in the direction whose components
 * along the crossed axes are reversed. */
static int pull_source(const orc_ctx* c, int x, int y, int z, int a, int64_t* src, int* asrc)
{
    int v[3] = {x - c->e[a][0], y - c->e[a][1], z - c->e[a][2]};
    const int pos[3] = {x, y, z};
    int wall = 0, open = 0, flip[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        if (v[d] >= 0 && v[d] < c->n[d]) continue;
        int face = 2 * d + (v[d] < 0 ? 0 : 1);
        int bc = c->p.bc[face];
        if (bc == BC_PERIODIC) v[d] = (v[d] + c->n[d]) % c->n[d];
        else if (bc == BC_WALL) wall = 1;
        else if (bc == BC_FREESLIP) { v[d] = pos[d]; flip[d] = 1; }
        else open = 1;
    }
    if (wall) return 1;
    if (open) return 2;
    *src = nid(c, v[0], v[1], v[2]);
    *asrc = a;
    if (flip[0] || flip[1] || flip[2]) {
        int m[3];
        for (int d = 0; d < 3; ++d) m[d] = flip[d] ? -c->e[a][d] : c->e[a][d];
        for (int b = 0; b < c->Q; ++b)
            if (c->e[b][0] == m[0] && c->e[b][1] == m[1] && c->e[b][2] == m[2]) *asrc = b;
    }
    return 0;
}

/* ------------------------------------------------------------ public API */

int orc_validate(const orc_params* p)
{
    if (p->lattice != ORC_D2Q9 && p->lattice != ORC_D3Q19) return -1;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
    if (p->lattice == ORC_D2Q9 && p->nz != 1) return -1;
    if (!(p->rho_L > 0 && p->rho_H > 0 && p->tau_H > 0 && p->mu_ratio >= 0)) return -1;
    if (!(p->mu_ratio > 0 || p->tau_L > 0)) return -1;
    /* an interface narrower than two lattice units is not resolved by the
     * isotropic stencils of eq:gradient_phi / eq:laplacian_phi */
    if (!(p->W >= 2 && p->mobility > 0 && p->sigma >= 0)) return -1;
    if (p->visc_model != 0 && p->visc_model != 1) return -1;
    int D = p->lattice == ORC_D2Q9 ? 2 : 3, L = D - 1;
    if (p->outlet_scheme < 0 || p->outlet_scheme > 2) return -1;
    for (int d = 0; d < D; ++d) {
        int lo = p->bc[2 * d], hi = p->bc[2 * d + 1];
        if (lo < 0 || lo > 4 || hi < 0 || hi > 4) return -1;
        if ((lo == BC_PERIODIC) != (hi == BC_PERIODIC)) return -1;
        if (lo == BC_OUTFLOW || hi == BC_INLET) return -1;
        int open_lo = lo == BC_INLET || lo == BC_OUTFLOW, open_hi = hi == BC_INLET || hi == BC_OUTFLOW;
        if (d != L && (open_lo || open_hi)) return -1;
    }
    int n[3] = {p->nx, p->ny, p->nz};
    int lo = p->bc[2 * L], hi = p->bc[2 * L + 1];
    if ((lo == BC_INLET || hi == BC_OUTFLOW) && n[L] < 4) return -1;
    /* what enters through the inlet must be able to leave: an inlet needs the
     * convective outlet on the opposite face (the paper's jet set-up, Sec. 6) */
    if (lo == BC_INLET && hi != BC_OUTFLOW) return -1;
    return 0;
}

orc_ctx* orc_create(const orc_params* p)
{
    if (orc_validate(p) != 0) return NULL;
    orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    if (!c) return NULL;
    c->p = *p;
    /* Reading R3: mu_X = rho_X tau_X c_s^2, so mu_H / mu_L = ratio gives
     * tau_L = tau_H (rho_H / rho_L) / ratio */
    if (p->mu_ratio > 0) c->p.tau_L = p->tau_H * (p->rho_H / p->rho_L) / p->mu_ratio;
    if (p->lattice == ORC_D2Q9) {      /* 2D: no z faces, no z force */
        c->p.bc[4] = c->p.bc[5] = BC_PERIODIC;
        c->p.force[2] = 0.0;
    }
    fill_lattice(c, p->lattice);
    if (invert(c->Q, c->M, c->Minv) != 0) { free(c); return NULL; }
    c->L = c->D - 1;
    c->n[0] = p->nx; c->n[1] = p->ny; c->n[2] = p->nz;
    c->N = (int64_t)p->nx * p->ny * p->nz;
    size_t sz = (size_t)c->N * c->Q * sizeof(double);
    c->fA = (double*)calloc(1, sz); c->gA = (double*)calloc(1, sz);
    c->fB = (double*)calloc(1, sz); c->gB = (double*)calloc(1, sz);
    c->fs = (double*)calloc(1, sz); c->gs = (double*)calloc(1, sz);
    c->phi = (double*)calloc((size_t)c->N, sizeof(double));
    if (!c->fA || !c->gA || !c->fB || !c->gB || !c->fs || !c->gs || !c->phi) {
        free(c->fA); free(c->gA); free(c->fB); free(c->gB); free(c->fs); free(c->gs); free(c->phi);
        free(c);
        return NULL;
    }
    return c;
}

void orc_destroy(orc_ctx* c)
{
    if (!c) return;
    free(c->fA); free(c->gA); free(c->fB); free(c->gB); free(c->fs); free(c->gs); free(c->phi);
    free(c);
}

/* Initial state: g_a = phi Gamma_a(u) (eq:equilibrium_function),
 * f_a = p* w_a + Gamma_a(u) - w_a (eq:equilibrium).  Inputs are the float32
 * fields handed to every implementation; u holds D planes; pstar may be NULL. */
void orc_init(orc_ctx* c, const float* phi, const float* u, const float* pstar)
{
    int Q = c->Q;
    for (int64_t i = 0; i < c->N; ++i) {
        double uu[3] = {0, 0, 0};
        for (int d = 0; d < c->D; ++d) uu[d] = u ? (double)u[(int64_t)d * c->N + i] : 0.0;
        double ps = pstar ? (double)pstar[i] : 0.0;
        double ph = (double)phi[i];
        for (int a = 0; a < Q; ++a) {
            double G = Gamma(c, a, uu);
            c->gA[i * Q + a] = ph * G;
            c->fA[i * Q + a] = ps * c->w[a] + (G - c->w[a]);
        }
    }
}

static void compute_phi(orc_ctx* c, const double* g)
{
    int Q = c->Q;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->N; ++i) {
        double s = 0.0;
        for (int a = 0; a < Q; ++a) s += g[i * Q + a];
        c->phi[i] = s;
    }
}

/* Outlet speed U at column (t0, t1) of the outlet: the first moment of f
 * along the outward normal at layer N-1 after streaming (Reading R9). */
static double outlet_speed(const orc_ctx* c, const double* fB, int t0, int t1)
{
    int L = c->L, Q = c->Q, nL = c->n[L];
    int64_t iM = (c->D == 2) ? nid(c, t0, nL - 2, 0) : nid(c, t0, t1, nL - 2);
    double U = 0.0;
    for (int a = 0; a < Q; ++a) U += fB[iM * Q + a] * c->e[a][L];
    return U;
}

/* Open-face rules of App. B applied to the post-streaming state B, given the
 * state A of the previous time level (the outlet reads chi(N, t) from A).
 *
 * Velocity inlet (f) and phase-field inlet (g), Reading R8.  The velocity
 * rule holds for f' = f + F/2 (eq:velocity_boundary_u,
 * eq:velocity_boundary_distribution with eq:force_term), with F the force
 * the next macroscopic update finds at the node: the interfacial forces
 * F_s, F_p, F_mu need derivatives of phi, which are not evaluated at the
 * inlet, so F = F_b = (rho - rho_ref) g (eq:gravity_force) with rho from
 * phi_in (eq:mass_conservation makes sum g = phi_in).  The known populations
 * are shifted to f', the unknown ones are formed in f' and shifted back.
 *
 * Convective outlet, eq:implicit_convective / eq:convective_f/g:
 * chi(N, t+1) = [chi(N, t) + lambda chi(N-1, t+1)] / (1 + lambda) for every
 * population of both sets, lambda = U dt/dy clamped to [0, 1]; U of
 * eq:velocity_options: local (outlet_speed), or its maximum or average over
 * the layer. */
static void apply_faces(const orc_ctx* c, const double* fA, const double* gA, double* fB, double* gB)
{
    int Q = c->Q, L = c->L;
    int nt0 = c->n[0], nt1 = (c->D == 3) ? c->n[1] : 1;
    if (c->p.bc[2 * L] == BC_INLET) {
        for (int t1 = 0; t1 < nt1; ++t1)
            for (int t0 = 0; t0 < nt0; ++t0) {
                int64_t i = (c->D == 2) ? nid(c, t0, 0, 0) : nid(c, t0, t1, 0);
                double* f = fB + i * Q;
                double* g = gB + i * Q;
                double phi_in, un;
                inlet_profile(c, t0, t1, &phi_in, &un);
                double uin[3] = {0, 0, 0};
                uin[L] = un;
                /* eq:density_interpolation (Reading R4), eq:gravity_force */
                double ph = phi_in < 0.0 ? 0.0 : (phi_in > 1.0 ? 1.0 : phi_in);
                double rho = c->p.rho_L + ph * (c->p.rho_H - c->p.rho_L);
                double F[3];
                for (int d = 0; d < 3; ++d) F[d] = (rho - c->p.rho_ref) * c->p.force[d];
                double half[QMAX], fp[QMAX];
                for (int a = 0; a < Q; ++a) {
                    double eF = 0.0;
                    for (int d = 0; d < 3; ++d) eF += c->e[a][d] * F[d];
                    half[a] = 0.5 * c->w[a] * eF / (rho * CS2);   /* F_a / 2, eq:force_term */
                    fp[a] = f[a] + half[a];
                }
                double Mt[3] = {0, 0, 0}, theta = 0.0;
                int ndiag = 0;
                for (int b = 0; b < Q; ++b) {
                    if (c->e[b][L] != 0) continue;          /* Lambda = {e.n = 0} */
                    double Gb = Gamma(c, b, uin);
                    /* f^eq_b = p* w_b + Gamma_b - w_b; the p* part sums to 0 over Lambda */
                    for (int d = 0; d < 3; ++d) Mt[d] += c->e[b][d] * (fp[b] - (Gb - c->w[b]));
                    theta += g[b] - phi_in * Gb;            /* eq:excess_density */
                }
                for (int a = 0; a < Q; ++a) {
                    if (c->e[a][L] <= 0) continue;
                    int tang = 0;
                    for (int d = 0; d < 3; ++d) if (d != L && c->e[a][d] != 0) tang = 1;
                    ndiag += tang;
                }
                for (int a = 0; a < Q; ++a) {
                    if (c->e[a][L] <= 0) continue;          /* unknown: e_a . n > 0 */
                    int ab = c->opp[a];
                    double Ga = Gamma(c, a, uin), Gab = Gamma(c, ab, uin);
                    double eM = 0.0;
                    int tang = 0;
                    for (int d = 0; d < 3; ++d) {
                        if (d == L) continue;
                        eM += c->e[a][d] * Mt[d];
                        if (c->e[a][d] != 0) tang = 1;
                    }
                    /* eq:velocity_boundary_distribution (p* cancels; tangential factor 1/2, R8) */
                    double fpa = fp[ab] + (Ga - Gab) - 0.5 * eM;
                    f[a] = fpa - half[a];
                    g[a] = phi_in * Ga - (g[ab] - phi_in * Gab) - (tang ? theta / ndiag : 0.0);
                }
            }
    }
    if (c->p.bc[2 * L + 1] == BC_OUTFLOW) {
        int nL = c->n[L];
        double Umax = -1e300, Usum = 0.0;
        for (int t1 = 0; t1 < nt1; ++t1)
            for (int t0 = 0; t0 < nt0; ++t0) {
                double U = outlet_speed(c, fB, t0, t1);
                if (U > Umax) Umax = U;
                Usum += U;
            }
        const double Uglob = c->p.outlet_scheme == 1 ? Umax : Usum / ((double)nt0 * nt1);
        for (int t1 = 0; t1 < nt1; ++t1)
            for (int t0 = 0; t0 < nt0; ++t0) {
                int64_t iN, iM;
                if (c->D == 2) { iN = nid(c, t0, nL - 1, 0); iM = nid(c, t0, nL - 2, 0); }
                else { iN = nid(c, t0, t1, nL - 1); iM = nid(c, t0, t1, nL - 2); }
                double U = c->p.outlet_scheme == 0 ? outlet_speed(c, fB, t0, t1) : Uglob;
                double lam = U < 0.0 ? 0.0 : (U > 1.0 ? 1.0 : U);
                for (int a = 0; a < Q; ++a) {
                    fB[iN * Q + a] = (fA[iN * Q + a] + lam * fB[iM * Q + a]) / (1.0 + lam);
                    gB[iN * Q + a] = (gA[iN * Q + a] + lam * gB[iM * Q + a]) / (1.0 + lam);
                }
            }
    }
}

/* One time step: macroscopic update + collision on the current state A,
 * pull streaming into B, inlet/outlet fix-ups on B, swap. */
static void step_once(orc_ctx* c)
{
    int Q = c->Q, nx = c->n[0], ny = c->n[1], nz = c->n[2];
    compute_phi(c, c->gA);

#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->N; ++i) {
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        double phin[QMAX];
        gather_phi(c, c->phi, x, y, z, phin);
        node_update(c, c->fA + i * Q, c->gA + i * Q, phin, is_inlet_node(c, x, y, z), c->fs + i * Q,
                    c->gs + i * Q, NULL, NULL);
    }

    /* eq:streaming_f/g with eq:periodic_f/g and eq:no_slip_f/g */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->N; ++i) {
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        for (int a = 0; a < Q; ++a) {
            int64_t s;
            int as;
            int k = pull_source(c, x, y, z, a, &s, &as);
            if (k == 0) {
                c->fB[i * Q + a] = c->fs[s * Q + as];
                c->gB[i * Q + a] = c->gs[s * Q + as];
            } else if (k == 1) {
                c->fB[i * Q + a] = c->fs[i * Q + c->opp[a]];
                c->gB[i * Q + a] = c->gs[i * Q + c->opp[a]];
            } else {
                c->fB[i * Q + a] = 0.0;   /* unknown: set by the open-face rule */
                c->gB[i * Q + a] = 0.0;
            }
        }
    }

    apply_faces(c, c->fA, c->gA, c->fB, c->gB);
    (void)nz;
    double* t;
    t = c->fA; c->fA = c->fB; c->fB = t;
    t = c->gA; c->gA = c->gB; c->gB = t;
}

void orc_step(orc_ctx* c, int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; ++s) step_once(c);
}

/* Advection of the phase field alone in a prescribed velocity field (the
 * circular interface in a shear flow of Sec. 5.3): eq:lbe_interface with the
 * forcing term eq:forcing_term (Reading R7) and g^eq = phi Gamma(u)
 * (eq:equilibrium_function) for the velocity u = scale * uf (uf: D planes
 * [nz][ny][nx], x fastest), then pull streaming of g (eq:streaming_g,
 * eq:periodic_g, eq:no_slip_g).  f is not changed.  Faces must be periodic
 * or walls (returns -1 otherwise). */
int orc_advect(orc_ctx* c, const double* uf, double scale, int64_t nsteps)
{
    int Q = c->Q, nx = c->n[0], ny = c->n[1];
    for (int f = 0; f < 2 * c->D; ++f)
        if (c->p.bc[f] != BC_PERIODIC && c->p.bc[f] != BC_WALL && c->p.bc[f] != BC_FREESLIP) return -1;
    const double tau_phi = c->p.mobility / CS2;
    for (int64_t step = 0; step < nsteps; ++step) {
        compute_phi(c, c->gA);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < c->N; ++i) {
            int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
            double phin[QMAX];
            gather_phi(c, c->phi, x, y, z, phin);
            const double* g = c->gA + i * Q;
            double phi = 0.0;
            for (int a = 0; a < Q; ++a) phi += g[a];
            double gphi[3] = {0, 0, 0};
            for (int a = 0; a < Q; ++a)
                for (int d = 0; d < 3; ++d) gphi[d] += c->w[a] * phin[a] * c->e[a][d] / CS2;   /* eq:gradient_phi */
            double gn = sqrt(gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2]);
            double nrm[3] = {0, 0, 0};
            if (gn >= 1e-12)
                for (int d = 0; d < 3; ++d) nrm[d] = gphi[d] / gn;
            double u[3] = {0, 0, 0};
            for (int d = 0; d < c->D; ++d) u[d] = scale * uf[(int64_t)d * c->N + i];
            for (int a = 0; a < Q; ++a) {
                double en = 0.0;
                for (int d = 0; d < 3; ++d) en += c->e[a][d] * nrm[d];
                double Fphi = (1.0 - 4.0 * (phi - 0.5) * (phi - 0.5)) / c->p.W * c->w[a] * en;
                double gbar = phi * Gamma(c, a, u) - 0.5 * Fphi;
                c->gs[i * Q + a] = g[a] - (g[a] - gbar) / (tau_phi + 0.5) + Fphi;
            }
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < c->N; ++i) {
            int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
            for (int a = 0; a < Q; ++a) {
                int64_t src;
                int as;
                int k = pull_source(c, x, y, z, a, &src, &as);
                c->gB[i * Q + a] = k == 0 ? c->gs[src * Q + as] : c->gs[i * Q + c->opp[a]];
            }
        }
        double* t = c->gA; c->gA = c->gB; c->gB = t;
    }
    return 0;
}

/* Macroscopic fields of the current state: phi, u (D planes), p = p* rho c_s^2.
 * Any output pointer may be NULL. */
void orc_fields(orc_ctx* c, double* phi, double* u, double* p)
{
    int Q = c->Q, nx = c->n[0], ny = c->n[1];
    compute_phi(c, c->gA);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->N; ++i) {
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
        double phin[QMAX], out[5];
        gather_phi(c, c->phi, x, y, z, phin);
        node_update(c, c->fA + i * Q, c->gA + i * Q, phin, is_inlet_node(c, x, y, z), NULL, NULL, out, NULL);
        if (phi) phi[i] = out[0];
        if (u) for (int d = 0; d < c->D; ++d) u[(int64_t)d * c->N + i] = out[1 + d];
        if (p) p[i] = out[4];
    }
}

/* Populations of the current state, population-major [a][node]. */
void orc_get_pops(const orc_ctx* c, double* f, double* g)
{
    for (int a = 0; a < c->Q; ++a)
        for (int64_t i = 0; i < c->N; ++i) {
            if (f) f[(int64_t)a * c->N + i] = c->fA[i * c->Q + a];
            if (g) g[(int64_t)a * c->N + i] = c->gA[i * c->Q + a];
        }
}

void orc_set_pops(orc_ctx* c, const double* f, const double* g)
{
    for (int a = 0; a < c->Q; ++a)
        for (int64_t i = 0; i < c->N; ++i) {
            c->fA[i * c->Q + a] = f[(int64_t)a * c->N + i];
            c->gA[i * c->Q + a] = g[(int64_t)a * c->N + i];
        }
}

/* The open-face rules alone (test hook for the pins of App. B): fB, gB are
 * a post-streaming state [a][node] (population-major); the context's current
 * state plays chi(N, t) of the outlet rule.  fB and gB are overwritten with
 * the state after the inlet and outlet rules. */
void orc_apply_faces(orc_ctx* c, double* fB, double* gB)
{
    int Q = c->Q;
    for (int a = 0; a < Q; ++a)
        for (int64_t i = 0; i < c->N; ++i) {
            c->fB[i * Q + a] = fB[(int64_t)a * c->N + i];
            c->gB[i * Q + a] = gB[(int64_t)a * c->N + i];
        }
    apply_faces(c, c->fA, c->gA, c->fB, c->gB);
    for (int a = 0; a < Q; ++a)
        for (int64_t i = 0; i < c->N; ++i) {
            fB[(int64_t)a * c->N + i] = c->fB[i * Q + a];
            gB[(int64_t)a * c->N + i] = c->gB[i * Q + a];
        }
}

/* --------------------------------------------------- exports for the pins */

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Velocity set, weights and opposite table of a lattice; returns Q. */
int orc_lattice(int lattice, int32_t* e, double* w, int32_t* opp)
{
    orc_ctx c;
    fill_lattice(&c, lattice);
    for (int a = 0; a < c.Q; ++a) {
        for (int d = 0; d < 3; ++d) if (e) e[a * 3 + d] = c.e[a][d];
        if (w) w[a] = c.w[a];
        if (opp) opp[a] = c.opp[a];
    }
    return c.Q;
}

/* The transformation matrix M (row-major Q x Q) as the oracle holds it. */
int orc_matrix(int lattice, double* M)
{
    orc_ctx c;
    fill_lattice(&c, lattice);
    for (int k = 0; k < c.Q; ++k)
        for (int a = 0; a < c.Q; ++a) M[k * c.Q + a] = c.M[k][a];
    return c.Q;
}

/* Dense collision matrix M^-1 S M (row-major) for a shear rate s_nu. */
int orc_collision_matrix(int lattice, double s_nu, double* C)
{
    orc_ctx c;
    fill_lattice(&c, lattice);
    if (invert(c.Q, c.M, c.Minv) != 0) return -1;
    for (int a = 0; a < c.Q; ++a) {
        double x[QMAX] = {0}, y[QMAX];
        x[a] = 1.0;
        apply_MSM(&c, s_nu, x, y);
        for (int b = 0; b < c.Q; ++b) C[b * c.Q + a] = y[b];
    }
    return c.Q;
}

/* One node in isolation: given its post-stream populations f, g and the
 * stencil values phin[a] = phi(x + e_a), return the post-collision
 * populations, {phi, u_x, u_y, u_z, p} and the intermediate terms listed at
 * node_update.  Uses the physical parameters of
 * ctx (its grid is ignored). */
void orc_collide_node(const orc_ctx* c, const double* f, const double* g, const double* phin,
                      double* fs, double* gs, double* out, double* terms)
{
    node_update(c, f, g, phin, 0, fs, gs, out, terms);
}

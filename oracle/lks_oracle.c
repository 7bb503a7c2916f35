/*
 * lks_oracle.c -- plain FP64 CPU implementation of the Lattice Kinetic Scheme (LKS)
 * state march and the Adjoint Lattice Kinetic Scheme (ALKS) of Tanabe, Yaji and
 * Ushijima, "Adjoint lattice kinetic scheme for topology optimization in fluid
 * problems" (arXiv 2411.03090).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is checked
 * against.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the CUDA
 * library, and it must never be reached from the product path.
 *
 * Everything is written as loops over nodes and lattice directions, in the order
 * the paper states the scheme, so that each line can be compared with the paper:
 *
 *   lattice            D2Q9, Eq. (D2Q9w); directions numbered so that the
 *                      opposite pairs of Eq. (ftilde) hold (2<->4, 5<->7, 6<->8)
 *   design             alpha_gamma Eq. (brinkman); K_gamma Eq. (conductivity);
 *                      nu <-> A Eq. (A); K <-> B Eq. (B)
 *   forward            Eqs. (rho), (u), (T) with f^eq Eq. (feq2), g^eq Eq. (geq2)
 *                      and the Brinkman correction Eq. (lbef_ex) taken implicitly
 *   forward BCs        Sec. 2.4 (prescribed u, prescribed p and u_s, T or flux)
 *   objective          Eq. (fj) with a domain integrand J_O (total dissipation,
 *                      plus an optional kappa_T * T term) plus kappa_p times the
 *                      static pressure drop J_p = sum_in p - sum_out p (Eq.
 *                      objective_pipebend, p = rho / 3, dGamma = 1, over the
 *                      inlet span and the outlet nodes) plus kappa_E times the
 *                      energy loss J_E = sum -n.u (p + |u|^2 / 2) over the same
 *                      nodes (Eq. objective_doublepipe)
 *   adjoint            Eqs. (ap)-(aq) with f~^eq Eq. (afeq), g~^eq Eq. (ageq) and
 *                      the sources of Eqs. (albef_ex), (albeg_ex) (App. A)
 *   adjoint BCs        Eq. (afboundaryu) solved in the least-squares sense as in
 *                      Sec. 2.5 (generalized inverse, residual Eq. (r_definition)),
 *                      with the boundary objective term on the inlet span and the
 *                      outlet (+-kappa_p per row: the derivative of the integrand
 *                      kappa_p p with respect to p; for J_E the same on the inlet,
 *                      and on the outlet three times its derivative with respect
 *                      to f_i through u_n);
 *                      the pressure, temperature and heat-flux versions of App. A
 *                      Eqs. (afboundaryp), (agboundaryT), (agboundaryq),
 *                      (afboundaryuq) by the same least-squares procedure
 *   sensitivity        the integrand of <J', dgamma> in Sec. 2.5
 *
 * Readings where the paper is silent (lattice units dx = dt = 1, so every
 * (1/eps) dx factor is one; implicit Brinkman; second-order central differences
 * inside and second-order one-sided differences on the domain edge; Zou-He-type
 * density / normal velocity on edges; corner rules; objective) are restated next
 * to the code they affect.
 *
 * The outlet row term of the energy loss (its kinetic part, the only part left
 * under the gauge-pressure reading) is pinned as arithmetic only: it equals three
 * times the derivative of the outlet integrand with respect to each population
 * (brute-force central differences in the test).  Its effect on the gradient lies
 * below what central differences of J resolve at the check geometry's velocities
 * (dropping it moves the ALKS / FD ratios by 3e-4).
 *
 * Storage: every field is an array of nx*ny doubles, node (i, j) at j*nx + i
 * (x fastest).  Node (i, j) sits at x = i, y = j; the domain edges carry nodes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* D2Q9 lattice, Eq. (D2Q9w)                                                  */
/* ------------------------------------------------------------------------- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Thermal edge condition kinds (Sec. 2.4). */
#define ORC_T_FIXED 0 /* T = T_bar                         */
#define ORC_T_FLUX 1  /* -q_alpha n_alpha = q_bar_w         */

/* Edge ids for the thermal table. */
#define ORC_LEFT 0
#define ORC_RIGHT 1
#define ORC_BOTTOM 2
#define ORC_TOP 3

/* Problem description.  The Python side mirrors this struct with ctypes. */
typedef struct {
    int nx, ny;
    double nu;                 /* kinematic viscosity; A from Eq. (A)          */
    double alpha_bar, q_alpha; /* Eq. (brinkman)                              */
    double u_max;              /* inlet peak velocity                         */
    double pulse_mean, pulse_amp, pulse_period; /* u_in(t) = u_max (mean + amp sin(2 pi t / period)) */
    int in_y0, in_y1;          /* inlet span on the left edge (inclusive)      */
    int out_y0, out_y1;        /* pressure-outlet span on the right edge      */
    double rho_out;            /* rho_bar = 3 p_bar at the outlet              */
    int thermal;               /* 1: march the thermal lattice as well        */
    double K_f, K_s, q_K;      /* Eq. (conductivity)                          */
    int t_kind[4];             /* per edge (left, right, bottom, top)         */
    double t_val[4];           /* T_bar or q_bar_w per edge                    */
    double kappa_T;            /* weight of the T term in J_O                  */
    double kappa_p;            /* weight of the static pressure drop J_p       */
    int periodic;              /* bit 0: x periodic (no left / right edges),
                                  bit 1: y periodic (no bottom / top edges)    */
    double G_x, G_y;           /* uniform external force G of Eq. (lbef_ex)   */
    double beta_bar, q_beta;   /* heat source Q = beta_gamma (1 - T), Eqs.
                                  (heatsource), (betagamma); beta_bar = 0: none */
    double kappa_Q;            /* weight of the heat-exchange objective
                                  -sum beta_gamma (1 - T), Eq. (objective_heatexchanger) */
    double gb_x, gb_y;         /* Boussinesq force G = g beta (T - T_ref),
                                  Eq. (boussinesqforce): the products g_a beta */
    double T_ref;
    int heat_x0, heat_x1;      /* heated segment of a flux-type bottom edge     */
    double heat_q;             /* its heat flux (replaces t_val[bottom] there)   */
    double kappa_E;            /* weight of the energy loss J_E, Eq.
                                  (objective_doublepipe)                          */
} orc_problem;

/* ------------------------------------------------------------------------- */
/* Material interpolation, Eqs. (brinkman), (conductivity), (A), (B)          */
/* ------------------------------------------------------------------------- */
static double lks_A(const orc_problem *p) { return (1.0 / 6.0 - p->nu) * 9.0 / 2.0; }

static double alpha_of(const orc_problem *p, double g) {
    return p->alpha_bar * p->q_alpha * (1.0 - g) / (p->q_alpha + g);
}
static double dalpha_of(const orc_problem *p, double g) {
    double d = p->q_alpha + g;
    return -p->alpha_bar * p->q_alpha * (1.0 + p->q_alpha) / (d * d);
}
static double K_of(const orc_problem *p, double g) {
    return p->K_f + (p->K_s - p->K_f) * p->q_K * (1.0 - g) / (p->q_K + g);
}
static double B_of(const orc_problem *p, double g) { return 3.0 * (1.0 / 6.0 - K_of(p, g)); }
/* Eq. (betagamma): beta_gamma = beta_bar q_beta (1 - gamma) / (q_beta + gamma) */
static double beta_of(const orc_problem *p, double g) {
    return p->beta_bar * p->q_beta * (1.0 - g) / (p->q_beta + g);
}
static double dbeta_of(const orc_problem *p, double g) {
    double d = p->q_beta + g;
    return -p->beta_bar * p->q_beta * (1.0 + p->q_beta) / (d * d);
}
static double dB_of(const orc_problem *p, double g) {
    double d = p->q_K + g;
    double dK = -(p->K_s - p->K_f) * p->q_K * (1.0 + p->q_K) / (d * d);
    return -3.0 * dK;
}

/* ------------------------------------------------------------------------- */
/* Geometry helpers                                                          */
/* ------------------------------------------------------------------------- */
#define AT(f, i, j) ((f)[(size_t)(j) * (size_t)nx + (size_t)(i)])

/* Maps (i, j) onto the lattice along periodic axes (wrap-around); returns 1 when
 * the node exists (always along a periodic axis). */
static int node_at(const orc_problem *p, int *i, int *j) {
    if (p->periodic & 1) *i = ((*i % p->nx) + p->nx) % p->nx;
    if (p->periodic & 2) *j = ((*j % p->ny) + p->ny) % p->ny;
    return *i >= 0 && *i < p->nx && *j >= 0 && *j < p->ny;
}

/* Node classes. */
enum { N_INTERIOR = 0, N_VELOCITY = 1, N_PRESSURE = 2, N_CORNER = 3 };

/* Classify node (i, j); writes the outward normal (sum of the two face normals at
 * a corner). */
static int classify(const orc_problem *p, int i, int j, int *nxo, int *nyo) {
    int nx = p->nx, ny = p->ny;
    int px = p->periodic & 1, py = p->periodic & 2;
    int left = !px && (i == 0), right = !px && (i == nx - 1);
    int bottom = !py && (j == 0), top = !py && (j == ny - 1);
    *nxo = (right ? 1 : 0) - (left ? 1 : 0);
    *nyo = (top ? 1 : 0) - (bottom ? 1 : 0);
    if ((left || right) && (bottom || top)) return N_CORNER;
    if (left || bottom || top) return N_VELOCITY;
    if (right) return (j >= p->out_y0 && j <= p->out_y1) ? N_PRESSURE : N_VELOCITY;
    return N_INTERIOR;
}

/* Thermal kind of an edge or corner node: corners follow the horizontal edge. */
static int thermal_edge(const orc_problem *p, int i, int j) {
    if (j == 0) return ORC_BOTTOM;
    if (j == p->ny - 1) return ORC_TOP;
    if (i == 0) return ORC_LEFT;
    return ORC_RIGHT;
}

/* Inlet profile: u_in(t) * parabola over the inlet span, zero elsewhere. */
static double inlet_u(const orc_problem *p, int j, double t) {
    if (j < p->in_y0 || j > p->in_y1) return 0.0;
    double H = (double)(p->in_y1 - p->in_y0);
    double y = (double)(j - p->in_y0);
    double amp = p->pulse_mean;
    if (p->pulse_period > 0.0) amp += p->pulse_amp * sin(2.0 * M_PI * t / p->pulse_period);
    return p->u_max * amp * 4.0 * y * (H - y) / (H * H);
}

/* ------------------------------------------------------------------------- */
/* Gradient operator: second-order central differences inside, second-order    */
/* one-sided differences on the domain edge (the same operator everywhere).    */
/* ------------------------------------------------------------------------- */
static double ddx(const orc_problem *p, const double *f, int i, int j) {
    int nx = p->nx;
    if (p->periodic & 1) return (AT(f, (i + 1) % nx, j) - AT(f, (i + nx - 1) % nx, j)) / 2.0;
    if (i == 0) return (-3.0 * AT(f, 0, j) + 4.0 * AT(f, 1, j) - AT(f, 2, j)) / 2.0;
    if (i == nx - 1) return (3.0 * AT(f, nx - 1, j) - 4.0 * AT(f, nx - 2, j) + AT(f, nx - 3, j)) / 2.0;
    return (AT(f, i + 1, j) - AT(f, i - 1, j)) / 2.0;
}
static double ddy(const orc_problem *p, const double *f, int i, int j) {
    int nx = p->nx, ny = p->ny;
    if (p->periodic & 2) return (AT(f, i, (j + 1) % ny) - AT(f, i, (j + ny - 1) % ny)) / 2.0;
    if (j == 0) return (-3.0 * AT(f, i, 0) + 4.0 * AT(f, i, 1) - AT(f, i, 2)) / 2.0;
    if (j == ny - 1) return (3.0 * AT(f, i, ny - 1) - 4.0 * AT(f, i, ny - 2) + AT(f, i, ny - 3)) / 2.0;
    return (AT(f, i, j + 1) - AT(f, i, j - 1)) / 2.0;
}

/* Velocity gradient entering f^eq at node (i, j): g = du/dx, du/dy, dv/dx, dv/dy.
 * The operator above everywhere, except the derivative of the normal velocity
 * component along the edge normal at edge nodes, which is taken from continuity,
 * Eq. (cont): du_n/dn = -du_s/ds with the derivative along the edge (central
 * differences along the edge; zero at corner nodes, where both edges carry a zero
 * tangential velocity).  The one-sided normal derivative of u_n makes the march
 * unstable for A < 0 (nu > 1/6); for the exact solutions the two agree. */
static void vel_grad(const orc_problem *p, const double *u, const double *v, int i, int j, double *g) {
    int nx = p->nx, ny = p->ny;
    g[0] = ddx(p, u, i, j);
    g[1] = ddy(p, u, i, j);
    g[2] = ddx(p, v, i, j);
    g[3] = ddy(p, v, i, j);
    int xe = !(p->periodic & 1) && (i == 0 || i == nx - 1);
    int ye = !(p->periodic & 2) && (j == 0 || j == ny - 1);
    if (xe && ye) {
        g[0] = 0.0;
        g[3] = 0.0;
    } else if (xe) {
        g[0] = -g[3];
    } else if (ye) {
        g[3] = -g[0];
    }
}

/* ------------------------------------------------------------------------- */
/* Equilibria                                                                 */
/* ------------------------------------------------------------------------- */
/* Eq. (feq2): f_k^eq = w_k { rho + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2
 *                           + A (du_a/dx_b + du_b/dx_a) c_a c_b }          */
static double feq(int k, double A, double rho, double u, double v, double dudx, double dudy,
                  double dvdx, double dvdy) {
    double cu = CX[k] * u + CY[k] * v;
    double S_xx = 2.0 * dudx, S_yy = 2.0 * dvdy, S_xy = dudy + dvdx;
    double Scc = S_xx * CX[k] * CX[k] + 2.0 * S_xy * CX[k] * CY[k] + S_yy * CY[k] * CY[k];
    return WT[k] * (rho + 3.0 * cu + 4.5 * cu * cu - 1.5 * (u * u + v * v) + A * Scc);
}

/* Eq. (geq2), read with the B-term linear in grad T:
 * g_k^eq = w_k [ T (1 + 3 c.u) + B c.grad T ]                               */
static double geq(int k, double T, double u, double v, double B, double dTdx, double dTdy) {
    double cu = CX[k] * u + CY[k] * v;
    return WT[k] * (T * (1.0 + 3.0 * cu) + B * (CX[k] * dTdx + CY[k] * dTdy));
}

/* ------------------------------------------------------------------------- */
/* Forward LKS step for one node                                              */
/* ------------------------------------------------------------------------- */
/* Computes the state at node (i, j) and time t from the state at time t-1.
 * out[0..3] = rho, u, v, T.  T is left at 0 when the thermal lattice is off. */
void orc_forward_node(const orc_problem *p, const double *gamma, double t, const double *rho,
                      const double *u, const double *v, const double *T, int i, int j,
                      double *out) {
    int nx = p->nx, ny = p->ny;
    double A = lks_A(p);
    int n_x, n_y;
    int cls = classify(p, i, j, &n_x, &n_y);

    /* Streamed populations f_k(x, t) = f_k^eq(x - c_k, t - 1) (Eq. lbef2), and
     * g_k likewise (Eq. lbeg2); known[k] = 0 where x - c_k is off the lattice. */
    double f[9], g[9];
    int known[9];
    for (int k = 0; k < 9; ++k) {
        int si = i - CX[k], sj = j - CY[k];
        known[k] = node_at(p, &si, &sj);
        f[k] = g[k] = 0.0;
        if (!known[k]) continue;
        double gu[4];
        vel_grad(p, u, v, si, sj, gu);
        f[k] = feq(k, A, AT(rho, si, sj), AT(u, si, sj), AT(v, si, sj), gu[0], gu[1], gu[2], gu[3]);
        if (p->thermal)
            g[k] = geq(k, AT(T, si, sj), AT(u, si, sj), AT(v, si, sj), B_of(p, AT(gamma, si, sj)),
                       ddx(p, T, si, sj), ddy(p, T, si, sj));
    }

    double r = 0.0, uu = 0.0, vv = 0.0, TT = 0.0;
    if (cls == N_INTERIOR) {
        /* Eqs. (rho), (u), (T); Brinkman and force terms of Eq. (lbef_ex), the
         * Brinkman term implicit: u = (u* + G) / (1 + alpha_gamma)  (sum of c_k
         * times Eq. lbef_ex, with sum_k w_k c_k c_k = 1/3).  The heat source of
         * Eq. (lbeg_ex) enters T once per step at t + dt, implicitly as the Brinkman
         * term: T = (T* + beta_gamma) / (1 + beta_gamma) for Q = beta_gamma (1 - T).
         * G = G0 + g beta (T - T_ref) uses that new T (Eq. boussinesqforce). */
        double us = 0.0, vs = 0.0;
        for (int k = 0; k < 9; ++k) {
            r += f[k];
            us += CX[k] * f[k];
            vs += CY[k] * f[k];
            TT += g[k];
        }
        double Gx = p->G_x, Gy = p->G_y;
        if (p->thermal) {
            if (p->beta_bar != 0.0) {
                double b = beta_of(p, AT(gamma, i, j));
                TT = (TT + b) / (1.0 + b);
            }
            Gx += p->gb_x * (TT - p->T_ref);
            Gy += p->gb_y * (TT - p->T_ref);
        }
        double a = alpha_of(p, AT(gamma, i, j));
        uu = (us + Gx) / (1.0 + a);
        vv = (vs + Gy) / (1.0 + a);
    } else if (cls == N_CORNER) {
        /* Corner: wall node, u = 0; density carried over from the previous step
         * of the edge neighbour at the same x (one row into the lattice). */
        int jn = (j == 0) ? 1 : ny - 2;
        r = AT(rho, i, jn);
        uu = vv = 0.0;
    } else {
        /* Edge node.  Sums over the known populations, split by c.n. */
        double s0 = 0.0, sp = 0.0; /* c.n == 0 and c.n > 0 (outgoing) */
        for (int k = 0; k < 9; ++k) {
            int cn = CX[k] * n_x + CY[k] * n_y;
            if (cn == 0) s0 += f[k];
            else if (cn > 0) sp += f[k];
        }
        if (cls == N_VELOCITY) {
            /* u = u_bar (walls: 0); rho from mass and normal momentum:
             * rho = sum_{c.n=0} f + 2 sum_{c.n>0} f - u.n                      */
            uu = (i == 0) ? inlet_u(p, j, t) : 0.0;
            vv = 0.0;
            r = s0 + 2.0 * sp - (uu * n_x + vv * n_y);
        } else {
            /* Pressure outlet: rho = rho_bar, u_s = 0,
             * u.n = sum_{c.n=0} f + 2 sum_{c.n>0} f - rho_bar                 */
            r = p->rho_out;
            double un = s0 + 2.0 * sp - p->rho_out;
            uu = un * n_x;
            vv = un * n_y;
        }
    }

    if (p->thermal && cls != N_INTERIOR) {
        int e = thermal_edge(p, i, j);
        if (p->t_kind[e] == ORC_T_FIXED) {
            TT = p->t_val[e];
        } else if (cls == N_CORNER) {
            /* flux-type corner: temperature carried over from the vertical neighbour */
            int jn = (j == 0) ? 1 : ny - 2;
            TT = AT(T, i, jn);
        } else {
            /* -q.n = q_bar with q = sum (c - u) g:  T (1 + u.n) = sum_0 g + 2 sum_+ g + q_bar;
             * q_bar = heat_q on the heated segment of the bottom edge */
            double s0 = 0.0, sp = 0.0;
            for (int k = 0; k < 9; ++k) {
                int cn = CX[k] * n_x + CY[k] * n_y;
                if (cn == 0) s0 += g[k];
                else if (cn > 0) sp += g[k];
            }
            double qb = p->t_val[e];
            if (e == ORC_BOTTOM && i >= p->heat_x0 && i <= p->heat_x1) qb = p->heat_q;
            TT = (s0 + 2.0 * sp + qb) / (1.0 + uu * n_x + vv * n_y);
        }
    }
    out[0] = r;
    out[1] = uu;
    out[2] = vv;
    out[3] = p->thermal ? TT : 0.0;
}

/* One forward step over the whole lattice: state(t-1) -> state(t). */
void orc_forward_step(const orc_problem *p, const double *gamma, double t, const double *rho,
                      const double *u, const double *v, const double *T, double *rho_n, double *u_n,
                      double *v_n, double *T_n) {
    int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double o[4];
            orc_forward_node(p, gamma, t, rho, u, v, T, i, j, o);
            AT(rho_n, i, j) = o[0];
            AT(u_n, i, j) = o[1];
            AT(v_n, i, j) = o[2];
            if (T_n) AT(T_n, i, j) = o[3];
        }
}

/* ------------------------------------------------------------------------- */
/* Objective: domain integrand J_O of Eq. (fj)                               */
/*   J_O = sum over interior nodes of                                        */
/*         nu/2 (S_xx^2 + 2 S_xy^2 + S_yy^2) + alpha_gamma |u|^2 + kappa_T T   */
/* ------------------------------------------------------------------------- */
/* Node (i, j), wrapped along periodic axes, and whether it is an interior node
 * (not on a domain edge; every node of a periodic axis is interior along it). */
static int is_interior(const orc_problem *p, int *i, int *j) {
    if (!node_at(p, i, j)) return 0;
    int xin = (p->periodic & 1) || (*i > 0 && *i < p->nx - 1);
    int yin = (p->periodic & 2) || (*j > 0 && *j < p->ny - 1);
    return xin && yin;
}

double orc_objective(const orc_problem *p, const double *gamma, const double *u, const double *v,
                     const double *T) {
    int nx = p->nx, ny = p->ny;
    double J = 0.0;
#pragma omp parallel for reduction(+ : J) schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int ii = i, jj = j;
            if (!is_interior(p, &ii, &jj)) continue;
            double Sxx = 2.0 * ddx(p, u, i, j), Syy = 2.0 * ddy(p, v, i, j);
            double Sxy = ddy(p, u, i, j) + ddx(p, v, i, j);
            double uu = AT(u, i, j), vv = AT(v, i, j);
            J += 0.5 * p->nu * (Sxx * Sxx + 2.0 * Sxy * Sxy + Syy * Syy) +
                 alpha_of(p, AT(gamma, i, j)) * (uu * uu + vv * vv);
            if (p->thermal) {
                J += p->kappa_T * AT(T, i, j);
                /* heat exchange, Eq. (objective_heatexchanger): -sum beta_gamma (1 - T) */
                if (p->kappa_Q != 0.0) J -= p->kappa_Q * beta_of(p, AT(gamma, i, j)) * (1.0 - AT(T, i, j));
            }
        }
    return J;
}

/* Inlet nodes: the velocity nodes of the left edge inside the inlet span (not the
 * corners); outlet nodes: the pressure nodes.  J_p = 1/3 (sum over inlet nodes of
 * rho - sum over outlet nodes of rho): Eq. objective_pipebend with p = rho / 3 and
 * dGamma = 1. */
static int is_inlet(const orc_problem *p, int i, int j) {
    return !(p->periodic & 1) && i == 0 && j > 0 && j < p->ny - 1 && j >= p->in_y0 && j <= p->in_y1;
}
double orc_pressure_drop(const orc_problem *p, const double *rho) {
    int nx = p->nx, ny = p->ny;
    double s = 0.0;
    if (p->periodic & 1) return 0.0; /* no inlet or outlet */
    for (int j = 1; j < ny - 1; ++j) {
        if (is_inlet(p, 0, j)) s += AT(rho, 0, j);
        if (j >= p->out_y0 && j <= p->out_y1) s -= AT(rho, nx - 1, j);
    }
    return s / 3.0;
}

/* Energy loss of one level, Eq. (objective_doublepipe): the flux of total pressure
 * out of the domain, sum over boundary nodes of -n.u (p + |u|^2 / 2) with dGamma = 1.
 * The walls carry u = 0, so the sum runs over the inlet nodes (n = (-1, 0):
 * -n.u = u) and the outlet nodes (n = (1, 0): -n.u = -u), the nodes of J_p.
 * Reading: p is the pressure above the outlet's, (rho - rho_bar) / 3.  A constant
 * added to p adds that constant times the net mass flux, which vanishes at steady
 * state, so the value is unchanged there and the outlet term keeps only its kinetic
 * part. */
double orc_energy_loss(const orc_problem *p, const double *rho, const double *u, const double *v) {
    int nx = p->nx, ny = p->ny;
    double s = 0.0;
    if (p->periodic & 1) return 0.0;
    for (int j = 1; j < ny - 1; ++j) {
        if (is_inlet(p, 0, j)) {
            double uu = AT(u, 0, j), vv = AT(v, 0, j);
            s += uu * ((AT(rho, 0, j) - p->rho_out) / 3.0 + 0.5 * (uu * uu + vv * vv));
        }
        if (j >= p->out_y0 && j <= p->out_y1) {
            double uu = AT(u, nx - 1, j), vv = AT(v, nx - 1, j);
            s -= uu * ((AT(rho, nx - 1, j) - p->rho_out) / 3.0 + 0.5 * (uu * uu + vv * vv));
        }
    }
    return s;
}

/* J = J_O + kappa_p J_p + kappa_E J_E of one level. */
double orc_objective_total(const orc_problem *p, const double *gamma, const double *rho,
                           const double *u, const double *v, const double *T) {
    double J = orc_objective(p, gamma, u, v, T);
    if (p->kappa_p != 0.0) J += p->kappa_p * orc_pressure_drop(p, rho);
    if (p->kappa_E != 0.0) J += p->kappa_E * orc_energy_loss(p, rho, u, v);
    return J;
}

/* dJ_O/du and dJ_O/dv at node (i, j): the derivative of the sum above, written
 * out term by term (S at an interior neighbour z depends on u(i, j) through the
 * central differences of z). */
/* S component `which` (0: S_xx, 1: S_xy, 2: S_yy) at the neighbour (i + di, j + dj)
 * when that neighbour is an interior node, else 0. */
static double S_nb(const orc_problem *p, const double *u, const double *v, int i, int j, int di, int dj,
                   int which) {
    int zi = i + di, zj = j + dj;
    if (!is_interior(p, &zi, &zj)) return 0.0;
    if (which == 0) return 2.0 * ddx(p, u, zi, zj);
    if (which == 2) return 2.0 * ddy(p, v, zi, zj);
    return ddy(p, u, zi, zj) + ddx(p, v, zi, zj);
}
void orc_dJdu_node(const orc_problem *p, const double *gamma, const double *u, const double *v,
                   int i, int j, double *ju, double *jv) {
    int nx = p->nx;
    double a = 0.0, b = 0.0;
    /* S_xx(z) = u(z+ex) - u(z-ex): z = (i-1,j) gives +S_xx(z), z = (i+1,j) gives -S_xx(z)  */
    a += S_nb(p, u, v, i, j, -1, 0, 0);
    a -= S_nb(p, u, v, i, j, +1, 0, 0);
    /* 2 S_xy^2 with S_xy(z) = (u(z+ey) - u(z-ey))/2 + ... : factor 2 * 1/2 = 1 */
    a += S_nb(p, u, v, i, j, 0, -1, 1);
    a -= S_nb(p, u, v, i, j, 0, +1, 1);
    b += S_nb(p, u, v, i, j, 0, -1, 2);
    b -= S_nb(p, u, v, i, j, 0, +1, 2);
    b += S_nb(p, u, v, i, j, -1, 0, 1);
    b -= S_nb(p, u, v, i, j, +1, 0, 1);
    a *= p->nu;
    b *= p->nu;
    int ii = i, jj = j;
    if (is_interior(p, &ii, &jj)) {
        double al = alpha_of(p, AT(gamma, i, j));
        a += 2.0 * al * AT(u, i, j);
        b += 2.0 * al * AT(v, i, j);
    }
    *ju = a;
    *jv = b;
}

/* ------------------------------------------------------------------------- */
/* Small dense least squares (normal equations, Gaussian elimination)         */
/* ------------------------------------------------------------------------- */
/* Minimise || M x - b ||_2 over x (m rows, n <= 8 columns).  Columns that are
 * identically zero do not enter the residual; they are set to zero, which is
 * the minimum-norm solution for them. */
static void lstsq_small(int m, int n, const double *M /* m x n, row major */, const double *b,
                        double *x) {
    double N[8][9];
    int live[8], nl = 0;
    for (int c = 0; c < n; ++c) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += fabs(M[r * n + c]);
        if (s > 0.0) live[nl++] = c;
        x[c] = 0.0;
    }
    for (int a = 0; a < nl; ++a) {
        for (int c = 0; c < nl; ++c) {
            double s = 0.0;
            for (int r = 0; r < m; ++r) s += M[r * n + live[a]] * M[r * n + live[c]];
            N[a][c] = s;
        }
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += M[r * n + live[a]] * b[r];
        N[a][nl] = s;
    }
    for (int c = 0; c < nl; ++c) { /* partial pivoting */
        int piv = c;
        for (int r = c + 1; r < nl; ++r)
            if (fabs(N[r][c]) > fabs(N[piv][c])) piv = r;
        if (piv != c)
            for (int q = 0; q <= nl; ++q) {
                double tmp = N[c][q];
                N[c][q] = N[piv][q];
                N[piv][q] = tmp;
            }
        for (int r = c + 1; r < nl; ++r) {
            double fct = N[r][c] / N[c][c];
            for (int q = c; q <= nl; ++q) N[r][q] -= fct * N[c][q];
        }
    }
    for (int c = nl - 1; c >= 0; --c) {
        double s = N[c][nl];
        for (int q = c + 1; q < nl; ++q) s -= N[c][q] * x[live[q]];
        x[live[c]] = s / N[c][c];
    }
}

/* Flow adjoint boundary condition at an edge node (Sec. 2.5 and App. A).
 * Residual for every direction i (Eq. r_definition, with dx = eps_f = 1):
 *   r_i = (n.c_i) f~_i - 2A sum_j w_j (n.c_j)(c_j.c_i) f~_j + m_i - kT (c_i.n)
 * where m_i = mu~.c_i on velocity nodes (Eq. afboundaryu) and
 *       m_i = lambda~ + mu~_s (c_i.s) on pressure nodes (Eq. afboundaryp),
 * and kT = kappa~ T on heat-flux edges (Eqs. afboundaryuq, afboundarypq).
 * The unknown f~_i are those whose gather point x + c_i is off the lattice; they
 * and the multipliers minimise ||r||_2 over all nine rows (generalized inverse).
 * f[] holds the known values on entry and all nine on exit.  mult[0..1] returns
 * the multipliers. */
void orc_bc_flow(int n_x, int n_y, int pressure, double A, double kT, const int *unknown,
                 double *f, double *mult, double jb, const double *jbv) {
    int U[9], nu_ = 0;
    for (int k = 0; k < 9; ++k)
        if (unknown[k]) U[nu_++] = k;
    int ncol = nu_ + 2;
    double Mfull[9][9];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            int cnc = CX[c] * n_x + CY[c] * n_y;
            double cc = (double)(CX[c] * CX[r] + CY[c] * CY[r]);
            Mfull[r][c] = (r == c ? (double)(CX[r] * n_x + CY[r] * n_y) : 0.0) - 2.0 * A * WT[c] * cnc * cc;
        }
    double Ms[9 * 8], rhs[9], x[8];
    int s_x = -n_y, s_y = n_x; /* tangent */
    for (int r = 0; r < 9; ++r) {
        for (int q = 0; q < nu_; ++q) Ms[r * ncol + q] = Mfull[r][U[q]];
        if (pressure) {
            Ms[r * ncol + nu_] = 1.0;
            Ms[r * ncol + nu_ + 1] = (double)(CX[r] * s_x + CY[r] * s_y);
        } else {
            Ms[r * ncol + nu_] = (double)CX[r];
            Ms[r * ncol + nu_ + 1] = (double)CY[r];
        }
        double s = 0.0;
        for (int c = 0; c < 9; ++c)
            if (!unknown[c]) s += Mfull[r][c] * f[c];
        s -= kT * (double)(CX[r] * n_x + CY[r] * n_y);
        rhs[r] = -s - jb - (jbv ? jbv[r] : 0.0);
    }
    lstsq_small(9, ncol, Ms, rhs, x);
    for (int q = 0; q < nu_; ++q) f[U[q]] = x[q];
    if (mult) {
        mult[0] = x[nu_];
        mult[1] = x[nu_ + 1];
    }
}

/* Thermal adjoint boundary condition (App. A):
 *   r_i = (n.c_i) g~_i - B sum_j w_j (n.c_j) g~_j + eta~              (Eq. agboundaryT)
 *   r_i = (n.c_i) g~_i - B sum_j w_j (n.c_j) g~_j + kappa~ (c_i - u).n (Eq. agboundaryq)
 * Least squares over all nine rows for the unknown g~ and the multiplier, which is
 * returned in *mult. */
void orc_bc_thermal(int n_x, int n_y, int flux, double B, double un, const int *unknown, double *g,
                    double *mult) {
    int U[9], nu_ = 0;
    for (int k = 0; k < 9; ++k)
        if (unknown[k]) U[nu_++] = k;
    int ncol = nu_ + 1;
    double Mfull[9][9];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            int cnc = CX[c] * n_x + CY[c] * n_y;
            Mfull[r][c] = (r == c ? (double)(CX[r] * n_x + CY[r] * n_y) : 0.0) - B * WT[c] * cnc;
        }
    double Ms[9 * 8], rhs[9], x[8];
    for (int r = 0; r < 9; ++r) {
        for (int q = 0; q < nu_; ++q) Ms[r * ncol + q] = Mfull[r][U[q]];
        Ms[r * ncol + nu_] = flux ? ((double)(CX[r] * n_x + CY[r] * n_y) - un) : 1.0;
        double s = 0.0;
        for (int c = 0; c < 9; ++c)
            if (!unknown[c]) s += Mfull[r][c] * g[c];
        rhs[r] = -s;
    }
    lstsq_small(9, ncol, Ms, rhs, x);
    for (int q = 0; q < nu_; ++q) g[U[q]] = x[q];
    if (mult) *mult = x[nu_];
}

/* ------------------------------------------------------------------------- */
/* ALKS step                                                                  */
/* ------------------------------------------------------------------------- */
/* Adjoint fields, in this order, each nx*ny: rho~, u~_x, u~_y, s~_xx, s~_xy, s~_yy,
 * T~, q~_x, q~_y.  (s~ is symmetric: s~_yx = s~_xy.) */
#define NADJ 9

/* Per-node equilibrium coefficients of the adjoint at level t+1 (Eqs. afeq, ageq):
 *   f~_k^eq = P + c_k . V   with  P = rho~,
 *   V_a = 3 (u~_a + 3 s~_ab u_b - rho~ u_a) - A d_b (s~_ab + s~_ba)
 *   g~^eq  = T~ + 3 q~.u - B div q~ - grad B . q~     (the same for every k)
 * using the state u at the same node and level. */
static void adjoint_eq_fields(const orc_problem *p, const double *gamma, const double *u,
                              const double *v, double *const *a, double *P, double *Vx, double *Vy,
                              double *G, double *Bfield) {
    int nx = p->nx, ny = p->ny;
    double A = lks_A(p);
    if (p->thermal) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) AT(Bfield, i, j) = B_of(p, AT(gamma, i, j));
    }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double rt = AT(a[0], i, j), ux = AT(a[1], i, j), uy = AT(a[2], i, j);
            double sxx = AT(a[3], i, j), sxy = AT(a[4], i, j), syy = AT(a[5], i, j);
            double uu = AT(u, i, j), vv = AT(v, i, j);
            double Dx = 2.0 * (ddx(p, a[3], i, j) + ddy(p, a[4], i, j));
            double Dy = 2.0 * (ddx(p, a[4], i, j) + ddy(p, a[5], i, j));
            AT(P, i, j) = rt;
            AT(Vx, i, j) = 3.0 * (ux + 3.0 * (sxx * uu + sxy * vv) - rt * uu) - A * Dx;
            AT(Vy, i, j) = 3.0 * (uy + 3.0 * (sxy * uu + syy * vv) - rt * vv) - A * Dy;
            if (p->thermal) {
                double qx = AT(a[7], i, j), qy = AT(a[8], i, j);
                double divq = ddx(p, a[7], i, j) + ddy(p, a[8], i, j);
                double dBx = ddx(p, Bfield, i, j), dBy = ddy(p, Bfield, i, j);
                AT(G, i, j) = AT(a[6], i, j) + 3.0 * (qx * uu + qy * vv) - AT(Bfield, i, j) * divq -
                              (dBx * qx + dBy * qy);
            }
        }
}

/* Exported form of the equilibrium coefficients above (P, V, G at every node). */
void orc_adjoint_eq(const orc_problem *p, const double *gamma, const double *u, const double *v,
                    double *const *a, double *P, double *Vx, double *Vy, double *G, double *Bwork) {
    adjoint_eq_fields(p, gamma, u, v, a, P, Vx, Vy, G, Bwork);
}

/* The row terms of the energy loss (Eq. objective_doublepipe) on an outlet node
 * with outward normal (n_x, n_y) and normal velocity un: there p = p_bar (the
 * gauge's zero) and u_s = 0, so the integrand is -un^3 / 2 with
 * un = sum_i (c_i . n) f_i / rho_bar, and row r carries three times its derivative
 * with respect to f_r (the scale of the pressure-drop row term, d/dp = 3 d/df_r). */
void orc_energy_outlet_rows(const orc_problem *p, double un, int n_x, int n_y, double *jbv) {
    double dJ = -1.5 * un * un;
    for (int r = 0; r < 9; ++r) jbv[r] = 3.0 * p->kappa_E * dJ * (double)(CX[r] * n_x + CY[r] * n_y) / p->rho_out;
}

/* Adjoint node update at level t from the equilibrium coefficients at level t+1
 * (already evaluated into P, Vx, Vy, G), the state at level t (u0, v0, T0) and
 * gamma.  out[0..8] in the adjoint field order.
 *
 * Interior nodes (Eqs. albef, albef_ex, albeg, albeg_ex, then the moments):
 *   f~_k = f~_k^eq(x + c_k) - 3 c_k.(alpha u~) + 3 T c_k.q~ - dJ_O/df_k
 *   g~_k = g~^eq(x + c_k) - dJ_O/dg_k
 * with dJ_O/df_k = c_k . dJ_O/du (J_O does not depend on rho) and
 * dJ_O/dg_k = dJ_O/dT = kappa_T; taking the moments, the Brinkman term is
 * implicit: u~ = (u~* - (1/3) dJ_O/du + T q~) / (1 + alpha_gamma).
 *
 * Edge nodes: the f~_k whose gather point is off the lattice follow from the
 * least-squares boundary rule; the moments of all nine are applied directly. */
void orc_adjoint_node(const orc_problem *p, const double *gamma, const double *P,
                      const double *Vx, const double *Vy, const double *G, const double *u0,
                      const double *v0, const double *T0, int i, int j, double *out) {
    int nx = p->nx;
    double A = lks_A(p);
    int n_x, n_y;
    int cls = classify(p, i, j, &n_x, &n_y);
    double f[9], g[9];
    int unknown[9];
    for (int k = 0; k < 9; ++k) {
        int gi = i + CX[k], gj = j + CY[k];
        unknown[k] = !node_at(p, &gi, &gj);
        f[k] = g[k] = 0.0;
        if (unknown[k]) continue;
        f[k] = AT(P, gi, gj) + CX[k] * AT(Vx, gi, gj) + CY[k] * AT(Vy, gi, gj);
        if (p->thermal) g[k] = AT(G, gi, gj);
    }
    if (cls != N_INTERIOR) {
        double kT = 0.0;
        if (p->thermal) {
            int e = thermal_edge(p, i, j);
            int flux = (p->t_kind[e] == ORC_T_FLUX);
            double un = AT(u0, i, j) * n_x + AT(v0, i, j) * n_y;
            double kap = 0.0;
            orc_bc_thermal(n_x, n_y, flux, B_of(p, AT(gamma, i, j)), un, unknown, g, &kap);
            if (flux) kT = kap * AT(T0, i, j);
        }
        /* boundary objective term of every row: d(kappa_p p)/dp, + on the inlet
         * and - on the outlet (reading: the row term is the derivative with
         * respect to p; with it the gradient matches central differences in the
         * paper's own pressure-drop verification, Sec. 2.6) */
        double jb = 0.0, jbv[9] = {0};
        if (cls == N_PRESSURE) jb = -p->kappa_p;
        else if (cls == N_VELOCITY && is_inlet(p, i, j)) jb = p->kappa_p;
        if (p->kappa_E != 0.0) {
            /* energy loss: on the inlet, the derivative of u (p + |u|^2 / 2) with
             * respect to p (u prescribed), as for J_p; on the outlet (p = p_bar, the
             * zero of the gauge, and u_s = 0) the integrand -u_n^3 / 2 depends on the
             * f_i through u_n = sum c_i.n f_i / rho_bar, and each row carries three
             * times d/df_i, the scale of the J_p row term (d/dp = 3 d/drho = 3 d/df_i). */
            if (cls == N_VELOCITY && is_inlet(p, i, j)) jb += p->kappa_E * AT(u0, i, j);
            if (cls == N_PRESSURE)
                orc_energy_outlet_rows(p, AT(u0, i, j) * n_x + AT(v0, i, j) * n_y, n_x, n_y, jbv);
        }
        orc_bc_flow(n_x, n_y, cls == N_PRESSURE, A, kT, unknown, f, NULL, jb, jbv);
    }
    double m[NADJ] = {0};
    for (int k = 0; k < 9; ++k) {
        m[0] += WT[k] * f[k];
        m[1] += WT[k] * CX[k] * f[k];
        m[2] += WT[k] * CY[k] * f[k];
        m[3] += WT[k] * CX[k] * CX[k] * f[k];
        m[4] += WT[k] * CX[k] * CY[k] * f[k];
        m[5] += WT[k] * CY[k] * CY[k] * f[k];
        m[6] += WT[k] * g[k];
        m[7] += WT[k] * CX[k] * g[k];
        m[8] += WT[k] * CY[k] * g[k];
    }
    if (cls == N_INTERIOR) {
        double ju, jv;
        orc_dJdu_node(p, gamma, u0, v0, i, j, &ju, &jv);
        double a = alpha_of(p, AT(gamma, i, j));
        double Tn = p->thermal ? AT(T0, i, j) : 0.0;
        m[1] = (m[1] - ju / 3.0 + Tn * m[7]) / (1.0 + a);
        m[2] = (m[2] - jv / 3.0 + Tn * m[8]) / (1.0 + a);
        if (p->thermal) {
            /* Eq. (albeg_ex): the source -dJ_O/dg_k = -dJ_O/dT; the Boussinesq term
             * 3 (dG_a/dg_k) u~_a = 3 g_a beta u~_a with u~ of this level; the heat
             * source term dQ/dg_k T~ = -beta_gamma T~ taken implicitly, as in the
             * forward step: T~ = (T~* + 3 g beta . u~ - dJ_O/dT) / (1 + beta_gamma). */
            double b = p->beta_bar != 0.0 ? beta_of(p, AT(gamma, i, j)) : 0.0;
            double dJdT = p->kappa_T + p->kappa_Q * b;
            m[6] = (m[6] + 3.0 * (p->gb_x * m[1] + p->gb_y * m[2]) - dJdT) / (1.0 + b);
        }
    }
    for (int q = 0; q < NADJ; ++q) out[q] = m[q];
}

/* One ALKS step over the lattice: adjoint(t+1) -> adjoint(t).
 * (u1, v1) is the state at t+1 (it enters f~^eq), (u0, v0, T0) the state at t.
 * a1 and a0 are arrays of NADJ field pointers.  work: 5*nx*ny doubles. */
void orc_adjoint_step(const orc_problem *p, const double *gamma, const double *u1,
                      const double *v1, const double *u0, const double *v0, const double *T0,
                      double *const *a1, double *const *a0, double *work) {
    int nx = p->nx, ny = p->ny;
    size_t N = (size_t)nx * ny;
    double *P = work, *Vx = work + N, *Vy = work + 2 * N, *G = work + 3 * N, *Bf = work + 4 * N;
    adjoint_eq_fields(p, gamma, u1, v1, a1, P, Vx, Vy, G, Bf);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double o[NADJ];
            orc_adjoint_node(p, gamma, P, Vx, Vy, G, u0, v0, T0, i, j, o);
            for (int q = 0; q < NADJ; ++q) AT(a0[q], i, j) = o[q];
        }
}

/* Sensitivity integrand at one level (Sec. 2.5), accumulated into sens:
 *   dJ_O/dgamma + 3 alpha' u.u~ - B' grad T . q~     (interior nodes)
 * with dJ_O/dgamma = alpha' |u|^2.  Edge nodes do not use gamma in the forward
 * scheme and receive nothing.  parts selects the terms: bit 0 the flow and
 * objective terms, bit 1 the thermal term.  In the unsteady sum the flow terms of
 * level t pair u(t) (which alpha_gamma scales in the step t-1 -> t) with u~(t),
 * for t = 1..n; the thermal term pairs grad T(t) (which B_gamma multiplies in the
 * step t -> t+1) with q~(t), for t = 0..n-1. */
void orc_sensitivity_parts(const orc_problem *p, const double *gamma, const double *u,
                           const double *v, const double *T, double *const *a, double *sens,
                           int parts) {
    int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int ii = i, jj = j;
            if (!is_interior(p, &ii, &jj)) continue;
            double gm = AT(gamma, i, j);
            double da = dalpha_of(p, gm);
            double uu = AT(u, i, j), vv = AT(v, i, j);
            double s = 0.0;
            if (parts & 1) s += da * (uu * uu + vv * vv) + 3.0 * da * (uu * AT(a[1], i, j) + vv * AT(a[2], i, j));
            if (p->thermal && p->beta_bar != 0.0 && (parts & 1)) {
                /* heat source and heat-exchange objective, paired with the level whose
                 * T they enter: -dQ/dgamma T~ - kappa_Q beta' (1 - T) */
                double db = dbeta_of(p, gm), Tv = AT(T, i, j);
                s += -db * (1.0 - Tv) * AT(a[6], i, j) - p->kappa_Q * db * (1.0 - Tv);
            }
            if (p->thermal && (parts & 2))
                s -= dB_of(p, gm) * (ddx(p, T, i, j) * AT(a[7], i, j) + ddy(p, T, i, j) * AT(a[8], i, j));
            AT(sens, i, j) += s;
        }
}

void orc_sensitivity_accum(const orc_problem *p, const double *gamma, const double *u,
                           const double *v, const double *T, double *const *a, double *sens) {
    orc_sensitivity_parts(p, gamma, u, v, T, a, sens, 3);
}

/* ------------------------------------------------------------------------- */
/* Drivers                                                                    */
/* ------------------------------------------------------------------------- */
void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Forward march of n_steps from the state at time t0 (arrays updated in place).
 * traj (optional): (n_steps + 1) * 3 * nx*ny doubles receiving u, v, T of every
 * level t0 .. t0 + n_steps.  J_acc (optional): adds J_O of every new level.
 * Returns max |u(t) - u(t-1)| of the last step. */
double orc_forward(const orc_problem *p, const double *gamma, int t0, int n_steps, double *rho,
                   double *u, double *v, double *T, double *traj, double *J_acc) {
    size_t N = (size_t)p->nx * p->ny;
    double *buf = (double *)calloc(4 * N, sizeof(double));
    double *r1 = buf, *u1 = buf + N, *v1 = buf + 2 * N, *T1 = buf + 3 * N;
    double res = 0.0;
    if (traj) {
        memcpy(traj + 0 * N, u, N * sizeof(double));
        memcpy(traj + 1 * N, v, N * sizeof(double));
        if (p->thermal) memcpy(traj + 2 * N, T, N * sizeof(double));
        else memset(traj + 2 * N, 0, N * sizeof(double));
    }
    for (int s = 1; s <= n_steps; ++s) {
        orc_forward_step(p, gamma, (double)(t0 + s), rho, u, v, p->thermal ? T : u, r1, u1, v1,
                         p->thermal ? T1 : NULL);
        res = 0.0;
        for (size_t q = 0; q < N; ++q) {
            double d = fabs(u1[q] - u[q]) + fabs(v1[q] - v[q]);
            if (d > res) res = d;
        }
        memcpy(rho, r1, N * sizeof(double));
        memcpy(u, u1, N * sizeof(double));
        memcpy(v, v1, N * sizeof(double));
        if (p->thermal) memcpy(T, T1, N * sizeof(double));
        if (traj) {
            double *lv = traj + (size_t)s * 3 * N;
            memcpy(lv, u, N * sizeof(double));
            memcpy(lv + N, v, N * sizeof(double));
            if (p->thermal) memcpy(lv + 2 * N, T, N * sizeof(double));
            else memset(lv + 2 * N, 0, N * sizeof(double));
        }
        if (J_acc) *J_acc += orc_objective_total(p, gamma, rho, u, v, T);
    }
    free(buf);
    return res;
}

/* Steady adjoint: n_iter ALKS steps with the state frozen at (u, v, T), starting
 * from zero (Eq. afinitial); the final adjoint fields are left in adj (NADJ*nx*ny,
 * field-major).  sens (nx*ny) receives the sensitivity of the final state.
 * Returns max |adjoint change| of the last iteration. */
double orc_steady_adjoint(const orc_problem *p, const double *gamma, const double *u,
                          const double *v, const double *T, int n_iter, double *adj,
                          double *sens) {
    size_t N = (size_t)p->nx * p->ny;
    double *other = (double *)calloc(NADJ * N, sizeof(double));
    double *work = (double *)calloc(5 * N, sizeof(double));
    double *Tz = NULL;
    if (!p->thermal) {
        Tz = (double *)calloc(N, sizeof(double));
        T = Tz;
    }
    memset(adj, 0, NADJ * N * sizeof(double));
    double *a1[NADJ], *a0[NADJ];
    double res = 0.0;
    for (int it = 0; it < n_iter; ++it) {
        double *src = (it % 2 == 0) ? adj : other, *dst = (it % 2 == 0) ? other : adj;
        for (int q = 0; q < NADJ; ++q) {
            a1[q] = src + q * N;
            a0[q] = dst + q * N;
        }
        orc_adjoint_step(p, gamma, u, v, u, v, T, a1, a0, work);
        res = 0.0;
        for (size_t q = 0; q < NADJ * N; ++q) {
            double d = fabs(dst[q] - src[q]);
            if (d > res) res = d;
        }
    }
    if (n_iter % 2 == 1) memcpy(adj, other, NADJ * N * sizeof(double));
    for (int q = 0; q < NADJ; ++q) a0[q] = adj + q * N;
    memset(sens, 0, N * sizeof(double));
    orc_sensitivity_accum(p, gamma, u, v, T, a0, sens);
    free(other);
    free(work);
    free(Tz);
    return res;
}

/* Unsteady adjoint over a stored trajectory traj (levels 0..n_steps, each u, v, T).
 * Terminal condition (Eqs. afinitial, aginitial): adjoint at level n_steps+1 is
 * zero; for t = n_steps .. 0 the ALKS step gives level t and the sensitivity terms
 * of level t are accumulated (flow terms for t >= 1, thermal term for t < n_steps).
 * adj receives the adjoint at level 0. */
void orc_unsteady_adjoint(const orc_problem *p, const double *gamma, int n_steps,
                          const double *traj, double *adj, double *sens) {
    size_t N = (size_t)p->nx * p->ny;
    double *other = (double *)calloc(NADJ * N, sizeof(double));
    double *work = (double *)calloc(5 * N, sizeof(double));
    double *a1[NADJ], *a0[NADJ];
    memset(adj, 0, NADJ * N * sizeof(double));
    memset(sens, 0, N * sizeof(double));
    double *cur = adj, *nxt = other; /* cur: level t+1 */
    for (int t = n_steps; t >= 0; --t) {
        const double *L1 = traj + (size_t)(t < n_steps ? t + 1 : t) * 3 * N;
        const double *L0 = traj + (size_t)t * 3 * N;
        for (int q = 0; q < NADJ; ++q) {
            a1[q] = cur + q * N;
            a0[q] = nxt + q * N;
        }
        orc_adjoint_step(p, gamma, L1, L1 + N, L0, L0 + N, L0 + 2 * N, a1, a0, work);
        orc_sensitivity_parts(p, gamma, L0, L0 + N, L0 + 2 * N, a0, sens,
                              (t >= 1 ? 1 : 0) | (t < n_steps ? 2 : 0));
        double *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (cur != adj) memcpy(adj, cur, NADJ * N * sizeof(double));
    free(other);
    free(work);
}

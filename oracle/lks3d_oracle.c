/*
 * lks3d_oracle.c -- plain FP64 CPU implementation of the three-dimensional (D3Q19)
 * form of the Lattice Kinetic Scheme (LKS) and its adjoint (ALKS) for a steady,
 * non-thermal duct: the scheme of arXiv 2411.03090 (Tanabe, Yaji, Ushijima)
 * carried to 19 velocities.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the oracle that the CUDA path is
 * checked against.  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper with
 * the CUDA library, and it must never be reached from the product path.
 *
 * The paper states the scheme in two dimensions (Sec. 2.4, 2.5 and App. A) and
 * names three dimensions as the natural extension (Sec. 4).  Every equation is
 * written here for D3Q19 exactly as the two-dimensional oracle writes it for D2Q9:
 *
 *   lattice            D3Q19: rest w = 1/3, six faces w = 1/18, twelve edges
 *                      w = 1/36; c_s^2 = 1/3 and the fourth-order isotropy that
 *                      makes nu = 1/6 - 2A/9 (Eq. A) hold unchanged
 *   forward            f_k^eq = w_k { rho + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2
 *                                     + A (du_a/dx_b + du_b/dx_a) c_a c_b }
 *                      (Eq. feq2 with three components), streamed
 *                      f_k(x) = f_k^eq(x - c_k), rho = sum f, u = sum c f / (1 + alpha)
 *   forward BCs        inlet face (x = 0): prescribed velocity; outlet face
 *                      (x = nx-1): prescribed pressure, tangential velocity zero;
 *                      the four side faces: walls (u = 0); nodes on two or three
 *                      faces: wall nodes with the density carried over
 *   objective          total dissipation J_O = sum over interior nodes of
 *                      nu/2 S:S + alpha_gamma |u|^2, plus kappa_p times the
 *                      static pressure drop J_p = sum_in p - sum_out p (Eq.
 *                      objective_pipebend, p = rho / 3, dGamma = 1) over the
 *                      inlet and outlet nodes that lie on one face only
 *   adjoint            f~_k = P(x + c_k) + c_k . V(x + c_k) with P = rho~ and
 *                      V_a = 3 (u~_a + 3 s~_ab u_b - rho~ u_a) - 2A d_b s~_ab
 *                      (Eq. afeq), moments rho~, u~ (3), s~ (6); implicit adjoint
 *                      Brinkman and the objective source (Eq. albef_ex)
 *   adjoint BCs        the generalized inverse of Sec. 2.5 (residual Eq.
 *                      r_definition) over all 19 rows, velocity multipliers
 *                      mu~ in R^3, pressure multipliers lambda~ and two tangential
 *                      mu~ (Eq. afboundaryp); the boundary objective enters every
 *                      row as +-kappa_p (inlet +, outlet -), the derivative of the
 *                      integrand kappa_p p with respect to p
 *   sensitivity        alpha' |u|^2 + 3 alpha' u . u~ at interior nodes (Sec. 2.5)
 *
 * Readings (restated at the code they affect): lattice units dx = dt = 1; implicit
 * Brinkman; second-order central differences inside and second-order one-sided
 * differences on the faces; on a node of exactly one face the normal derivative of
 * the normal velocity is taken from continuity (minus the two tangential
 * divergence terms), on nodes of two or three faces those derivatives are zero;
 * Zou-He-type density / normal velocity on faces; the inlet profile.
 *
 * Storage: every field is an array of nx*ny*nz doubles, node (i, j, k) at
 * (k*ny + j)*nx + i (x fastest).  The faces carry nodes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* D3Q19 lattice                                                              */
/* ------------------------------------------------------------------------- */
#define Q3 19
static const int C3[Q3][3] = {
    {0, 0, 0},                                                              /* rest  */
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1}, /* faces */
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},                        /* edges */
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W3[Q3] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                              1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* Tables exported for the lattice pins (isotropy, projection onto D2Q9). */
void orc3_lattice(int *c /* 19 x 3 */, double *w /* 19 */) {
    for (int q = 0; q < Q3; ++q) {
        for (int a = 0; a < 3; ++a) c[3 * q + a] = C3[q][a];
        w[q] = W3[q];
    }
}

typedef struct {
    int nx, ny, nz;
    double nu;
    double alpha_bar, q_alpha;
    double u_max;
    double rho_out;
    int profile; /* inlet: 0 duct (product of parabolas), 1 plane channel (parabola in y) */
    double kappa_p; /* weight of the static pressure drop in the objective */
} orc3_problem;

static double lks_A3(const orc3_problem *p) { return (1.0 / 6.0 - p->nu) * 9.0 / 2.0; }
/* Eq. (brinkman): alpha_gamma = alpha_bar q (1 - gamma) / (q + gamma) */
static double alpha3(const orc3_problem *p, double g) {
    return p->alpha_bar * p->q_alpha * (1.0 - g) / (p->q_alpha + g);
}
static double dalpha3(const orc3_problem *p, double g) {
    return -p->alpha_bar * p->q_alpha * (1.0 + p->q_alpha) / ((p->q_alpha + g) * (p->q_alpha + g));
}

#define A3(f, i, j, k) ((f)[((size_t)(k) * (size_t)ny + (size_t)(j)) * (size_t)nx + (size_t)(i)])

static int inside3(int nx, int ny, int nz, int i, int j, int k) {
    return i >= 0 && i < nx && j >= 0 && j < ny && k >= 0 && k < nz;
}

/* Node classes. */
#define M_INTERIOR 0
#define M_VELOCITY 1 /* inlet face and the four walls */
#define M_PRESSURE 2 /* outlet face */
#define M_CORNER 3   /* nodes on two or three faces: walls */

/* Outward normal n (sum of the face normals) and class of node (i, j, k). */
static int classify3(const orc3_problem *p, int i, int j, int k, int *n) {
    n[0] = (i == 0) ? -1 : (i == p->nx - 1 ? 1 : 0);
    n[1] = (j == 0) ? -1 : (j == p->ny - 1 ? 1 : 0);
    n[2] = (k == 0) ? -1 : (k == p->nz - 1 ? 1 : 0);
    int faces = abs(n[0]) + abs(n[1]) + abs(n[2]);
    if (faces == 0) return M_INTERIOR;
    if (faces >= 2) return M_CORNER;
    if (n[0] == 1) return M_PRESSURE;
    return M_VELOCITY;
}

/* Inlet velocity on the face x = 0 (zero on its edges, which are wall nodes). */
static double inlet3(const orc3_problem *p, int j, int k) {
    double y = (double)j / (double)(p->ny - 1), z = (double)k / (double)(p->nz - 1);
    if (p->profile == 1) return p->u_max * 4.0 * y * (1.0 - y);
    return p->u_max * 16.0 * y * (1.0 - y) * z * (1.0 - z);
}

/* ------------------------------------------------------------------------- */
/* Gradient operator: central differences inside, second-order one-sided on   */
/* the faces of the differentiated axis.                                      */
/* ------------------------------------------------------------------------- */
static double d3(const double *f, int nx, int ny, int nz, int i, int j, int k, int axis) {
    int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    int at = axis == 0 ? i : (axis == 1 ? j : k);
    int di = axis == 0, dj = axis == 1, dk = axis == 2;
    if (at == 0)
        return (-3.0 * A3(f, i, j, k) + 4.0 * A3(f, i + di, j + dj, k + dk) -
                A3(f, i + 2 * di, j + 2 * dj, k + 2 * dk)) / 2.0;
    if (at == n - 1)
        return (3.0 * A3(f, i, j, k) - 4.0 * A3(f, i - di, j - dj, k - dk) +
                A3(f, i - 2 * di, j - 2 * dj, k - 2 * dk)) / 2.0;
    return (A3(f, i + di, j + dj, k + dk) - A3(f, i - di, j - dj, k - dk)) / 2.0;
}

/* Velocity gradient g[a][b] = du_a/dx_b at node (i, j, k).  On a node of exactly
 * one face with normal axis a, du_a/dx_a comes from continuity (Eq. cont):
 * -(sum of the other two diagonal terms).  On nodes of two or three faces the
 * normal derivatives of the normal components are zero (the tangential velocity
 * vanishes along both walls). */
static void vel_grad3(const double *const *u, int nx, int ny, int nz, int i, int j, int k,
                      double g[3][3]) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) g[a][b] = d3(u[a], nx, ny, nz, i, j, k, b);
    int on[3] = {i == 0 || i == nx - 1, j == 0 || j == ny - 1, k == 0 || k == nz - 1};
    int faces = on[0] + on[1] + on[2];
    if (faces == 1) {
        int a = on[0] ? 0 : (on[1] ? 1 : 2);
        double s = 0.0;
        for (int b = 0; b < 3; ++b)
            if (b != a) s += g[b][b];
        g[a][a] = -s;
    } else if (faces >= 2) {
        for (int a = 0; a < 3; ++a)
            if (on[a]) g[a][a] = 0.0;
    }
}

/* Eq. (feq2) in three dimensions. */
static double feq3(int q, double A, double rho, const double *u, double g[3][3]) {
    double cu = 0.0, uu = 0.0, Scc = 0.0;
    for (int a = 0; a < 3; ++a) {
        cu += C3[q][a] * u[a];
        uu += u[a] * u[a];
        for (int b = 0; b < 3; ++b) Scc += C3[q][a] * C3[q][b] * (g[a][b] + g[b][a]);
    }
    return W3[q] * (rho + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu + A * Scc);
}

/* Moments of the equilibrium at one node, for the pins: out[0] = sum f,
 * out[1..3] = sum c f, out[4..9] = sum c_a c_b f (xx, xy, xz, yy, yz, zz). */
void orc3_feq_moments(double A, double rho, const double *u, const double *grad /* 9, g[a][b] */,
                      double *out) {
    double g[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) g[a][b] = grad[3 * a + b];
    for (int m = 0; m < 10; ++m) out[m] = 0.0;
    static const int PA[6] = {0, 0, 0, 1, 1, 2}, PB[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < Q3; ++q) {
        double f = feq3(q, A, rho, u, g);
        out[0] += f;
        for (int a = 0; a < 3; ++a) out[1 + a] += C3[q][a] * f;
        for (int m = 0; m < 6; ++m) out[4 + m] += C3[q][PA[m]] * C3[q][PB[m]] * f;
    }
}

/* ------------------------------------------------------------------------- */
/* Forward LKS step for one node                                              */
/* ------------------------------------------------------------------------- */
/* State at node (i, j, k) from the state of the previous step.  u[0..2] are the
 * velocity component arrays.  out[0..3] = rho, u, v, w. */
void orc3_forward_node(const orc3_problem *p, const double *gamma, const double *rho,
                       const double *const *u, int i, int j, int k, double *out) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double A = lks_A3(p);
    int n[3];
    int cls = classify3(p, i, j, k, n);
    double f[Q3];
    for (int q = 0; q < Q3; ++q) {
        int si = i - C3[q][0], sj = j - C3[q][1], sk = k - C3[q][2];
        f[q] = 0.0;
        if (!inside3(nx, ny, nz, si, sj, sk)) continue;
        double g[3][3], us[3];
        vel_grad3(u, nx, ny, nz, si, sj, sk, g);
        for (int a = 0; a < 3; ++a) us[a] = A3(u[a], si, sj, sk);
        f[q] = feq3(q, A, A3(rho, si, sj, sk), us, g);
    }
    double r = 0.0, uo[3] = {0.0, 0.0, 0.0};
    if (cls == M_INTERIOR) {
        double us[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < Q3; ++q) {
            r += f[q];
            for (int a = 0; a < 3; ++a) us[a] += C3[q][a] * f[q];
        }
        double al = alpha3(p, A3(gamma, i, j, k));
        for (int a = 0; a < 3; ++a) uo[a] = us[a] / (1.0 + al);
    } else if (cls == M_CORNER) {
        /* Wall node on two or three faces: u = 0; density carried over from the
         * previous step of the neighbour one node inward along the side-wall
         * normals (y and z), at the same x. */
        int jn = j + (j == 0 ? 1 : (j == ny - 1 ? -1 : 0));
        int kn = k + (k == 0 ? 1 : (k == nz - 1 ? -1 : 0));
        r = A3(rho, i, jn, kn);
    } else {
        double s0 = 0.0, sp = 0.0; /* c.n == 0 and c.n > 0 over the known f */
        for (int q = 0; q < Q3; ++q) {
            int cn = C3[q][0] * n[0] + C3[q][1] * n[1] + C3[q][2] * n[2];
            if (cn == 0) s0 += f[q];
            else if (cn > 0) sp += f[q];
        }
        if (cls == M_VELOCITY) {
            /* rho = sum_{c.n=0} f + 2 sum_{c.n>0} f - u.n */
            if (n[0] == -1) uo[0] = inlet3(p, j, k);
            r = s0 + 2.0 * sp - (uo[0] * n[0] + uo[1] * n[1] + uo[2] * n[2]);
        } else {
            /* outlet: rho = rho_bar, tangential u = 0,
             * u.n = sum_{c.n=0} f + 2 sum_{c.n>0} f - rho_bar */
            r = p->rho_out;
            double un = s0 + 2.0 * sp - p->rho_out;
            for (int a = 0; a < 3; ++a) uo[a] = un * n[a];
        }
    }
    out[0] = r;
    out[1] = uo[0];
    out[2] = uo[1];
    out[3] = uo[2];
}

void orc3_forward_step(const orc3_problem *p, const double *gamma, const double *rho,
                       const double *u, const double *v, const double *w, double *rho_n, double *u_n,
                       double *v_n, double *w_n) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    const double *uv[3] = {u, v, w};
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double o[4];
                orc3_forward_node(p, gamma, rho, uv, i, j, k, o);
                A3(rho_n, i, j, k) = o[0];
                A3(u_n, i, j, k) = o[1];
                A3(v_n, i, j, k) = o[2];
                A3(w_n, i, j, k) = o[3];
            }
}

/* ------------------------------------------------------------------------- */
/* Objective: J_O = sum over interior nodes of nu/2 S:S + alpha_gamma |u|^2     */
/* ------------------------------------------------------------------------- */
static int interior3(int nx, int ny, int nz, int i, int j, int k) {
    return i > 0 && j > 0 && k > 0 && i < nx - 1 && j < ny - 1 && k < nz - 1;
}

/* S_ab = du_a/dx_b + du_b/dx_a (central differences at interior nodes). */
static double S3(const double *const *u, int nx, int ny, int nz, int i, int j, int k, int a, int b) {
    return d3(u[a], nx, ny, nz, i, j, k, b) + d3(u[b], nx, ny, nz, i, j, k, a);
}

double orc3_objective(const orc3_problem *p, const double *gamma, const double *u, const double *v,
                      const double *w) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    const double *uv[3] = {u, v, w};
    double J = 0.0;
#pragma omp parallel for collapse(2) reduction(+ : J) schedule(static)
    for (int k = 1; k < nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                double SS = 0.0, uu = 0.0;
                for (int a = 0; a < 3; ++a) {
                    uu += A3(uv[a], i, j, k) * A3(uv[a], i, j, k);
                    for (int b = 0; b < 3; ++b) {
                        double s = S3(uv, nx, ny, nz, i, j, k, a, b);
                        SS += s * s;
                    }
                }
                J += 0.5 * p->nu * SS + alpha3(p, A3(gamma, i, j, k)) * uu;
            }
    return J;
}

/* Static pressure drop (Eq. objective_pipebend) with p = rho / 3 and dGamma = 1:
 *   J_p = 1/3 (sum over inlet nodes of rho - sum over outlet nodes of rho),
 * the inlet and outlet nodes being those of the faces x = 0 and x = nx-1 that lie on
 * no other face (the face edges are wall nodes). */
double orc3_pressure_drop(const orc3_problem *p, const double *rho) {
    int nx = p->nx, ny = p->ny;
    double s = 0.0;
    for (int k = 1; k < p->nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j) s += A3(rho, 0, j, k) - A3(rho, nx - 1, j, k);
    return s / 3.0;
}

/* J = J_O + kappa_p J_p of one level. */
double orc3_objective_total(const orc3_problem *p, const double *gamma, const double *rho,
                            const double *u, const double *v, const double *w) {
    double J = orc3_objective(p, gamma, u, v, w);
    if (p->kappa_p != 0.0) J += p->kappa_p * orc3_pressure_drop(p, rho);
    return J;
}

/* dJ_O/du_a at node (i, j, k), term by term: u_a(x) enters S_ad of the interior
 * neighbours x -+ e_d through their central differences, giving
 *   nu sum_d [ S_ad(x - e_d) - S_ad(x + e_d) ]  (+ 2 alpha u_a at interior x). */
void orc3_dJdu_node(const orc3_problem *p, const double *gamma, const double *const *u, int i,
                    int j, int k, double *ju) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int d = 0; d < 3; ++d) {
            int di = d == 0, dj = d == 1, dk = d == 2;
            if (interior3(nx, ny, nz, i - di, j - dj, k - dk)) s += S3(u, nx, ny, nz, i - di, j - dj, k - dk, a, d);
            if (interior3(nx, ny, nz, i + di, j + dj, k + dk)) s -= S3(u, nx, ny, nz, i + di, j + dj, k + dk, a, d);
        }
        s *= p->nu;
        if (interior3(nx, ny, nz, i, j, k)) s += 2.0 * alpha3(p, A3(gamma, i, j, k)) * A3(u[a], i, j, k);
        ju[a] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* Least squares (normal equations, Gaussian elimination with pivoting)       */
/* ------------------------------------------------------------------------- */
/* Minimise || M x - b ||_2 (m <= 19 rows, n <= 16 columns).  Identically zero
 * columns do not enter the residual and are set to zero. */
static void lstsq3(int m, int n, const double *M, const double *b, double *x) {
    double N[16][17];
    int live[16], nl = 0;
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
    for (int c = 0; c < nl; ++c) {
        int piv = c;
        for (int r = c + 1; r < nl; ++r)
            if (fabs(N[r][c]) > fabs(N[piv][c])) piv = r;
        if (piv != c)
            for (int q = 0; q <= nl; ++q) {
                double t = N[c][q];
                N[c][q] = N[piv][q];
                N[piv][q] = t;
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

/* Flow adjoint boundary rule at a face, box-edge or corner node.  Residual for
 * every direction r (Eq. r_definition with dx = 1, and the boundary objective term
 * of Eqs. afboundaryu / afboundaryp):
 *   r_r = (n.c_r) f~_r - 2A sum_j w_j (n.c_j)(c_j.c_r) f~_j + m_r + jb
 * with m_r = mu~ . c_r on velocity nodes (three multipliers) and
 *      m_r = lambda~ + mu~_1 (c_r.t_1) + mu~_2 (c_r.t_2) on the outlet face (t_1,
 *      t_2 the face's tangents).
 * The unknown f~ (gather point off the lattice) and the multipliers minimise
 * ||r||_2 over all 19 rows.  jb = dJ_dO/df_k, the same for every k (the boundary
 * objective depends on the f only through rho).  f[] holds the known values on
 * entry and all 19 on exit; mult[0..2] receives the multipliers. */
void orc3_bc_flow(const int *n, int pressure, double A, const int *unknown, double *f,
                  double *mult, double jb) {
    int U[Q3], nu_ = 0;
    for (int q = 0; q < Q3; ++q)
        if (unknown[q]) U[nu_++] = q;
    int ncol = nu_ + 3;
    double M[Q3][Q3];
    for (int r = 0; r < Q3; ++r)
        for (int c = 0; c < Q3; ++c) {
            int cnc = C3[c][0] * n[0] + C3[c][1] * n[1] + C3[c][2] * n[2];
            double cc = (double)(C3[c][0] * C3[r][0] + C3[c][1] * C3[r][1] + C3[c][2] * C3[r][2]);
            int cnr = C3[r][0] * n[0] + C3[r][1] * n[1] + C3[r][2] * n[2];
            M[r][c] = (r == c ? (double)cnr : 0.0) - 2.0 * A * W3[c] * cnc * cc;
        }
    /* tangents of a face with normal along one axis */
    int ax = n[0] != 0 ? 0 : (n[1] != 0 ? 1 : 2);
    int t1 = (ax + 1) % 3, t2 = (ax + 2) % 3;
    double Ms[Q3 * 16], rhs[Q3], x[16];
    for (int r = 0; r < Q3; ++r) {
        for (int q = 0; q < nu_; ++q) Ms[r * ncol + q] = M[r][U[q]];
        if (pressure) {
            Ms[r * ncol + nu_] = 1.0;
            Ms[r * ncol + nu_ + 1] = (double)C3[r][t1];
            Ms[r * ncol + nu_ + 2] = (double)C3[r][t2];
        } else {
            for (int a = 0; a < 3; ++a) Ms[r * ncol + nu_ + a] = (double)C3[r][a];
        }
        double s = 0.0;
        for (int c = 0; c < Q3; ++c)
            if (!unknown[c]) s += M[r][c] * f[c];
        rhs[r] = -s - jb;
    }
    lstsq3(Q3, ncol, Ms, rhs, x);
    for (int q = 0; q < nu_; ++q) f[U[q]] = x[q];
    if (mult)
        for (int a = 0; a < 3; ++a) mult[a] = x[nu_ + a];
}

/* ------------------------------------------------------------------------- */
/* ALKS step                                                                  */
/* ------------------------------------------------------------------------- */
/* Adjoint fields, in this order, each nx*ny*nz: rho~, u~_x, u~_y, u~_z,
 * s~_xx, s~_xy, s~_xz, s~_yy, s~_yz, s~_zz (s~ symmetric). */
#define NADJ3 10
static const int SA[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}}; /* index of s~_ab */

/* Per-node equilibrium coefficients of the adjoint at level t+1 (Eq. afeq):
 *   f~_k^eq = P + c_k . V,  P = rho~,
 *   V_a = 3 (u~_a + 3 s~_ab u_b - rho~ u_a) - A d_b (s~_ab + s~_ba)
 * with the state u at the same node and level.  PV: 4 arrays (P, Vx, Vy, Vz). */
void orc3_adjoint_eq(const orc3_problem *p, const double *const *u, const double *const *a,
                     double *const *PV) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double A = lks_A3(p);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double rt = A3(a[0], i, j, k);
                double us[3];
                for (int b = 0; b < 3; ++b) us[b] = A3(u[b], i, j, k);
                A3(PV[0], i, j, k) = rt;
                for (int c = 0; c < 3; ++c) {
                    double su = 0.0, D = 0.0;
                    for (int b = 0; b < 3; ++b) {
                        su += A3(a[SA[c][b]], i, j, k) * us[b];
                        D += 2.0 * d3(a[SA[c][b]], nx, ny, nz, i, j, k, b);
                    }
                    A3(PV[1 + c], i, j, k) = 3.0 * (A3(a[1 + c], i, j, k) + 3.0 * su - rt * us[c]) - A * D;
                }
            }
}

/* Adjoint node update at level t from the coefficients PV of level t+1, the state
 * at level t (u0) and gamma.  Interior: f~_k = f~_k^eq(x + c_k) - 3 c_k.(alpha u~)
 * - c_k . dJ_O/du (Eq. albef_ex with the objective source); the moments give
 * u~ = (u~* - (1/3) dJ_O/du) / (1 + alpha_gamma) (implicit).  Face, box-edge and
 * corner nodes: the unknown f~ from the least-squares rule, moments of all 19. */
void orc3_adjoint_node(const orc3_problem *p, const double *gamma, const double *const *PV,
                       const double *const *u0, int i, int j, int k, double *out) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    double A = lks_A3(p);
    int n[3];
    int cls = classify3(p, i, j, k, n);
    double f[Q3];
    int unknown[Q3];
    for (int q = 0; q < Q3; ++q) {
        int gi = i + C3[q][0], gj = j + C3[q][1], gk = k + C3[q][2];
        unknown[q] = !inside3(nx, ny, nz, gi, gj, gk);
        f[q] = 0.0;
        if (unknown[q]) continue;
        f[q] = A3(PV[0], gi, gj, gk);
        for (int a = 0; a < 3; ++a) f[q] += C3[q][a] * A3(PV[1 + a], gi, gj, gk);
    }
    if (cls != M_INTERIOR) {
        /* boundary objective term of every row: d(kappa_p p)/dp, + on the inlet and
         * - on the outlet (reading: the row term is the derivative with respect
         * to p; with it the gradient matches central differences in the paper's
         * own pressure-drop verification, Sec. 2.6) */
        double jb = 0.0;
        if (cls == M_PRESSURE) jb = -p->kappa_p;
        else if (cls == M_VELOCITY && n[0] == -1) jb = p->kappa_p;
        orc3_bc_flow(n, cls == M_PRESSURE, A, unknown, f, NULL, jb);
    }
    double m[NADJ3] = {0};
    for (int q = 0; q < Q3; ++q) {
        m[0] += W3[q] * f[q];
        for (int a = 0; a < 3; ++a) m[1 + a] += W3[q] * C3[q][a] * f[q];
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b) m[SA[a][b]] += W3[q] * C3[q][a] * C3[q][b] * f[q];
    }
    if (cls == M_INTERIOR) {
        double ju[3];
        orc3_dJdu_node(p, gamma, u0, i, j, k, ju);
        double al = alpha3(p, A3(gamma, i, j, k));
        for (int a = 0; a < 3; ++a) m[1 + a] = (m[1 + a] - ju[a] / 3.0) / (1.0 + al);
    }
    for (int q = 0; q < NADJ3; ++q) out[q] = m[q];
}

/* One ALKS step: adjoint(t+1) -> adjoint(t).  u1: state at t+1 (enters f~^eq),
 * u0: state at t.  a1, a0: NADJ3 field pointers.  work: 4*N doubles. */
void orc3_adjoint_step(const orc3_problem *p, const double *gamma, const double *const *u1,
                       const double *const *u0, const double *const *a1, double *const *a0,
                       double *work) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
    size_t N = (size_t)nx * ny * nz;
    double *PV[4] = {work, work + N, work + 2 * N, work + 3 * N};
    orc3_adjoint_eq(p, u1, a1, PV);
    const double *PVc[4] = {PV[0], PV[1], PV[2], PV[3]};
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double o[NADJ3];
                orc3_adjoint_node(p, gamma, PVc, u0, i, j, k, o);
                for (int q = 0; q < NADJ3; ++q) A3(a0[q], i, j, k) = o[q];
            }
}

/* Sensitivity integrand of one level at interior nodes (Sec. 2.5):
 *   dJ_O/dgamma + 3 alpha' u.u~ with dJ_O/dgamma = alpha' |u|^2. */
void orc3_sensitivity_accum(const orc3_problem *p, const double *gamma, const double *const *u,
                            const double *const *a, double *sens) {
    int nx = p->nx, ny = p->ny, nz = p->nz;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 1; k < nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                double da = dalpha3(p, A3(gamma, i, j, k));
                double uu = 0.0, ua = 0.0;
                for (int b = 0; b < 3; ++b) {
                    double ub = A3(u[b], i, j, k);
                    uu += ub * ub;
                    ua += ub * A3(a[1 + b], i, j, k);
                }
                A3(sens, i, j, k) += da * uu + 3.0 * da * ua;
            }
}

/* ------------------------------------------------------------------------- */
/* Drivers                                                                    */
/* ------------------------------------------------------------------------- */
/* Forward march of n_steps (arrays updated in place).  traj (optional):
 * (n_steps + 1) * 3 * N doubles receiving u, v, w of every level.  J_acc
 * (optional): adds J_O of every new level.  Returns max |du| of the last step. */
double orc3_forward(const orc3_problem *p, const double *gamma, int n_steps, double *rho, double *u,
                    double *v, double *w, double *traj, double *J_acc) {
    size_t N = (size_t)p->nx * p->ny * p->nz;
    double *buf = (double *)calloc(4 * N, sizeof(double));
    double *r1 = buf, *u1 = buf + N, *v1 = buf + 2 * N, *w1 = buf + 3 * N;
    double res = 0.0;
    if (traj) {
        memcpy(traj, u, N * sizeof(double));
        memcpy(traj + N, v, N * sizeof(double));
        memcpy(traj + 2 * N, w, N * sizeof(double));
    }
    for (int s = 1; s <= n_steps; ++s) {
        orc3_forward_step(p, gamma, rho, u, v, w, r1, u1, v1, w1);
        res = 0.0;
        for (size_t q = 0; q < N; ++q) {
            double d = fabs(u1[q] - u[q]) + fabs(v1[q] - v[q]) + fabs(w1[q] - w[q]);
            if (d > res) res = d;
        }
        memcpy(rho, r1, N * sizeof(double));
        memcpy(u, u1, N * sizeof(double));
        memcpy(v, v1, N * sizeof(double));
        memcpy(w, w1, N * sizeof(double));
        if (traj) {
            double *lv = traj + (size_t)s * 3 * N;
            memcpy(lv, u, N * sizeof(double));
            memcpy(lv + N, v, N * sizeof(double));
            memcpy(lv + 2 * N, w, N * sizeof(double));
        }
        if (J_acc) *J_acc += orc3_objective_total(p, gamma, rho, u, v, w);
    }
    free(buf);
    return res;
}

/* Steady adjoint: n_iter ALKS steps on the frozen state (u, v, w) from zero
 * (Eq. afinitial); adj (NADJ3*N) receives the final adjoint, sens (N) the
 * sensitivity.  Returns max |adjoint change| of the last iteration. */
double orc3_steady_adjoint(const orc3_problem *p, const double *gamma, const double *u,
                           const double *v, const double *w, int n_iter, double *adj, double *sens) {
    size_t N = (size_t)p->nx * p->ny * p->nz;
    double *other = (double *)calloc(NADJ3 * N, sizeof(double));
    double *work = (double *)calloc(4 * N, sizeof(double));
    const double *uv[3] = {u, v, w};
    memset(adj, 0, NADJ3 * N * sizeof(double));
    const double *a1[NADJ3];
    double *a0[NADJ3];
    double res = 0.0;
    for (int it = 0; it < n_iter; ++it) {
        double *src = (it % 2 == 0) ? adj : other, *dst = (it % 2 == 0) ? other : adj;
        for (int q = 0; q < NADJ3; ++q) {
            a1[q] = src + q * N;
            a0[q] = dst + q * N;
        }
        orc3_adjoint_step(p, gamma, uv, uv, a1, a0, work);
        res = 0.0;
        for (size_t q = 0; q < NADJ3 * N; ++q) {
            double d = fabs(dst[q] - src[q]);
            if (d > res) res = d;
        }
    }
    if (n_iter % 2 == 1) memcpy(adj, other, NADJ3 * N * sizeof(double));
    for (int q = 0; q < NADJ3; ++q) a1[q] = adj + q * N;
    memset(sens, 0, N * sizeof(double));
    orc3_sensitivity_accum(p, gamma, uv, a1, sens);
    free(other);
    free(work);
    return res;
}

/* Unsteady adjoint over a stored trajectory (levels 0..n_steps of u, v, w): the
 * adjoint at level n_steps+1 is zero; for t = n_steps .. 1 the ALKS step gives
 * level t and the sensitivity of level t is accumulated (J = sum_{t=1..n} J_O). */
void orc3_unsteady_adjoint(const orc3_problem *p, const double *gamma, int n_steps,
                           const double *traj, double *adj, double *sens) {
    size_t N = (size_t)p->nx * p->ny * p->nz;
    double *other = (double *)calloc(NADJ3 * N, sizeof(double));
    double *work = (double *)calloc(4 * N, sizeof(double));
    const double *a1[NADJ3];
    double *a0[NADJ3];
    memset(adj, 0, NADJ3 * N * sizeof(double));
    memset(sens, 0, N * sizeof(double));
    double *cur = adj, *nxt = other;
    for (int t = n_steps; t >= 1; --t) {
        const double *L1 = traj + (size_t)(t < n_steps ? t + 1 : t) * 3 * N;
        const double *L0 = traj + (size_t)t * 3 * N;
        const double *u1[3] = {L1, L1 + N, L1 + 2 * N};
        const double *u0[3] = {L0, L0 + N, L0 + 2 * N};
        for (int q = 0; q < NADJ3; ++q) {
            a1[q] = cur + q * N;
            a0[q] = nxt + q * N;
        }
        orc3_adjoint_step(p, gamma, u1, u0, a1, a0, work);
        orc3_sensitivity_accum(p, gamma, u0, (const double *const *)a0, sens);
        double *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (cur != adj) memcpy(adj, cur, NADJ3 * N * sizeof(double));
    free(other);
    free(work);
}

/*
 * Plain FP64 CPU oracle for the pseudopotential MRT lattice Boltzmann step of
 * Shan et al., "Pseudopotential MRT lattice Boltzmann model for cavitation
 * bubble collapse with high density ratio" (arXiv:1605.01800).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call this file:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or table with the CUDA library.
 *
 * It is slow on purpose: every step of one time update is a separate plain
 * sweep over the lattice in the order the paper writes the scheme.
 *
 *   sweep A  density  rho = sum_a f_a                       (Sec. 2.1, after Eq. 4)
 *            pseudopotential psi(rho)                        (Eq. 13 with the CS EOS, Eq. 15)
 *   sweep B  per fluid node: force F                        (Eq. 7)
 *            velocity v = (sum_a e_a f_a + F/2)/rho          (Eq. 6)
 *            m = M f, m_eq                                   (Eq. 3, Eq. 4)
 *            source S with Li's terms                        (Eq. 14)
 *            m* = m - Lambda (m - m_eq) + (I - Lambda/2) S   (Eq. 3, Lambda of Eq. 2)
 *            f* = M^-1 m*                                    (after Eq. 5)
 *   sweep C  streaming f_a(x + e_a) = f*_a(x)                (Eq. 5), periodic wrap,
 *            no-slip halfway bounce-back at solid nodes      (Sec. 4.1)
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *  - c = delta_t = delta_x = 1 and c_s^2 = 1/3 (standard D2Q9, makes Eq. 4 the
 *    moment equilibrium).
 *  - M is the orthogonal D2Q9 moment matrix whose rows are ordered
 *    (rho, e, zeta, j_x, q_x, j_y, q_y, p_xx, p_xy), the order fixed by Eq. 4
 *    and Eq. 8; velocities are numbered as the weights of Eq. 7
 *    (1-4 axis, 5-8 diagonal).
 *  - tau_varsigma of Eq. 14 is tau_zeta of Eq. 2.
 *  - psi^2 < 0 (density above the root of p_EOS = rho c_s^2) is clamped to 0
 *    and reported through the returned flags.
 *  - A solid neighbour in the force sum of Eq. 7 takes the psi of the fluid
 *    node being updated (neutral wetting).
 *  - In Eq. 14 the ratio |F|^2/psi^2 at psi = 0 takes its limit G^2 |g|^2,
 *    where F = -G psi g.
 *
 * Array layout: f[a][y][x], a = 0..8, x fastest, nx*ny nodes per plane.
 *
 * Threads: the three sweeps update every node from read-only inputs and
 * write disjoint outputs, so they may run their node loops on several
 * threads (OpenMP, oracle_set_threads; one thread unless asked) with
 * bitwise the same result. The mass sum stays serial, in node order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

/* Discrete velocities e_a, numbered as the weights of Eq. 7. */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Index of -e_a. */
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* Interaction weights of Eq. 7: w_1..4 = 1/3, w_5..8 = 1/12. */
static const double WINT[Q] = {0.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0,
                               1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0, 1.0 / 12.0};
static const double CS2 = 1.0 / 3.0;

/* Threads of the sweeps' node loops (1: serial). */
static int g_threads = 1;

void oracle_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int oracle_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* Flags returned by the oracle. */
#define OR_FLAG_PSI_CLAMPED 1u
#define OR_FLAG_NONFINITE 2u

typedef struct {
    int nx, ny;
    double a, b, R, T, G; /* Eq. 15 constants and the interaction strength of Eq. 7 / Eq. 13 */
    double s[Q];          /* diagonal of Lambda, Eq. 2, order (rho,e,zeta,j,q,j,q,nu,nu) */
    double eps;           /* epsilon of Eq. 14 */
    const unsigned char* solid; /* nx*ny, 1 = solid node; NULL = none */
    int eos;              /* psi: 0 Eq. 13 with CS (Eq. 15), 1 Eq. 13 with van der Waals,
                             2 Eq. 13 with Peng-Robinson, 3 Eq. 12 */
    double omega;         /* Peng-Robinson acentric factor */
} oracle_params;

/* ---- moment matrix, Sec. 2.1 ------------------------------------------ */

/* Row k of M evaluated at velocity (ex, ey): the polynomial definitions of
 * the nine D2Q9 moments. */
static double m_row(int k, int ex, int ey) {
    double e2 = (double)(ex * ex + ey * ey);
    switch (k) {
    case 0: return 1.0;                                   /* density        */
    case 1: return -4.0 + 3.0 * e2;                       /* energy e       */
    case 2: return 4.0 - 10.5 * e2 + 4.5 * e2 * e2;       /* energy^2 zeta  */
    case 3: return (double)ex;                            /* j_x            */
    case 4: return (-5.0 + 3.0 * e2) * ex;                /* q_x            */
    case 5: return (double)ey;                            /* j_y            */
    case 6: return (-5.0 + 3.0 * e2) * ey;                /* q_y            */
    case 7: return (double)(ex * ex - ey * ey);           /* p_xx           */
    default: return (double)(ex * ey);                    /* p_xy           */
    }
}

static double Mmat[Q][Q];
static double Minv[Q][Q];
static int mats_ready = 0;

/* M from its row polynomials; M^-1 = M^T D^-1 with D = diag(M M^T), which
 * holds because the rows of M are mutually orthogonal (Sec. 2.1). */
static void build_mats(void) {
    if (mats_ready) return;
    double d[Q];
    for (int k = 0; k < Q; ++k) {
        d[k] = 0.0;
        for (int a = 0; a < Q; ++a) {
            Mmat[k][a] = m_row(k, EX[a], EY[a]);
            d[k] += Mmat[k][a] * Mmat[k][a];
        }
    }
    for (int a = 0; a < Q; ++a)
        for (int k = 0; k < Q; ++k) Minv[a][k] = Mmat[k][a] / d[k];
    mats_ready = 1;
}

void oracle_moment_matrix(double* m_out, double* minv_out) {
    build_mats();
    for (int k = 0; k < Q; ++k)
        for (int a = 0; a < Q; ++a) {
            if (m_out) m_out[k * Q + a] = Mmat[k][a];
            if (minv_out) minv_out[k * Q + a] = Minv[k][a];
        }
}

/* ---- thermodynamics ---------------------------------------------------- */

/* Peng-Robinson temperature factor alpha(T) = (1 + k (1 - sqrt(T/Tc)))^2,
 * k = 0.37464 + 1.54226 omega - 0.26992 omega^2; Tc follows from the PR
 * constants a = 0.45724 R^2 Tc^2 / pc and b = 0.0778 R Tc / pc. */
static double pr_alpha(const oracle_params* P) {
    double Tc = (0.0778 / 0.45724) * P->a / (P->b * P->R);
    double k = 0.37464 + 1.54226 * P->omega - 0.26992 * P->omega * P->omega;
    double s = 1.0 + k * (1.0 - sqrt(P->T / Tc));
    return s * s;
}

/* psi of Eq. 12 (the first strategy): exp(-1/rho) for e = 0, else
 * (rho / (e + rho))^(1/e), where e = -G eps is the exponent of the
 * mechanical stability condition (Eq. 9) that Li's term with eps yields
 * (Li et al. 2013: e = -16 G sigma with 0.75 eps = 12 sigma; e = eps at the
 * paper's G = -1). */
static double psi_eq12(const oracle_params* P, double rho) {
    double e = -P->G * P->eps;
    if (e == 0.0) return exp(-1.0 / rho);
    return pow(rho / (e + rho), 1.0 / e);
}

/* Non-ideal LB pressure, Eq. 10 (c = 1). */
double oracle_pressure(const oracle_params* P, double rho, double psi) {
    return rho * CS2 + 0.5 * P->G * psi * psi;
}

/* The EOS: Carnahan-Starling (Eq. 15, the paper's), van der Waals or
 * Peng-Robinson for Eq. 13; for the Eq. 12 psi the EOS the model produces,
 * Eq. 10. */
double oracle_p_eos(const oracle_params* P, double rho) {
    double RT = P->R * P->T;
    switch (P->eos) {
    case 1: /* van der Waals */
        return rho * RT / (1.0 - P->b * rho) - P->a * rho * rho;
    case 2: /* Peng-Robinson */
        return rho * RT / (1.0 - P->b * rho) -
               P->a * pr_alpha(P) * rho * rho / (1.0 + 2.0 * P->b * rho - P->b * P->b * rho * rho);
    case 3: /* Eq. 12 psi in Eq. 10 */
        return oracle_pressure(P, rho, psi_eq12(P, rho));
    default: { /* Carnahan-Starling, Eq. 15 */
        double eta = P->b * rho / 4.0;
        double num = 1.0 + eta + eta * eta - eta * eta * eta;
        double den = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
        return rho * RT * num / den - P->a * rho * rho;
    }
    }
}

/* Pseudopotential (c = 1): Eq. 12 for eos 3, else the square root of Eq. 13.
 * Sets *flag on clamping or a non-finite value. */
double oracle_psi(const oracle_params* P, double rho, unsigned* flag) {
    if (P->eos == 3) {
        double v = rho > 0.0 ? psi_eq12(P, rho) : NAN;
        if (!isfinite(v)) {
            if (flag) *flag |= OR_FLAG_NONFINITE;
            return 0.0;
        }
        return v;
    }
    double arg = 2.0 * (oracle_p_eos(P, rho) - rho * CS2) / P->G;
    if (!isfinite(arg)) {
        if (flag) *flag |= OR_FLAG_NONFINITE;
        return 0.0;
    }
    if (arg < 0.0) {
        if (flag) *flag |= OR_FLAG_PSI_CLAMPED;
        return 0.0;
    }
    return sqrt(arg);
}

/* ---- helpers ----------------------------------------------------------- */

static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

static int is_solid(const oracle_params* P, int x, int y) {
    return P->solid != NULL && P->solid[(size_t)y * P->nx + x] != 0;
}

/* ---- force, Eq. 7 ------------------------------------------------------ */

/* F at node (x, y) from a psi field psi[y][x]. A solid neighbour contributes
 * the psi of the node itself. */
static void force_at(const oracle_params* P, const double* psi, int x, int y,
                     double* Fx, double* Fy, double* g2) {
    int nx = P->nx, ny = P->ny;
    double psi0 = psi[(size_t)y * nx + x];
    double gx = 0.0, gy = 0.0;
    for (int a = 1; a < Q; ++a) {
        int xn = wrap(x + EX[a], nx), yn = wrap(y + EY[a], ny);
        double pn = is_solid(P, xn, yn) ? psi0 : psi[(size_t)yn * nx + xn];
        gx += WINT[a] * pn * EX[a];
        gy += WINT[a] * pn * EY[a];
    }
    *Fx = -P->G * psi0 * gx;
    *Fy = -P->G * psi0 * gy;
    if (g2) *g2 = gx * gx + gy * gy;
}

/* Force field from a given psi field (exported so that Eq. 7 can be checked
 * on its own). Solid nodes get F = 0. */
void oracle_force_from_psi(const oracle_params* P, const double* psi, double* Fx,
                           double* Fy) {
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            size_t i = (size_t)y * P->nx + x;
            if (is_solid(P, x, y)) {
                Fx[i] = 0.0;
                Fy[i] = 0.0;
            } else {
                force_at(P, psi, x, y, &Fx[i], &Fy[i], NULL);
            }
        }
}

/* ---- equilibrium, Eq. 4 ------------------------------------------------ */

static void m_equilibrium(double rho, double vx, double vy, double* meq) {
    double v2 = vx * vx + vy * vy;
    meq[0] = rho;
    meq[1] = rho * (-2.0 + 3.0 * v2);
    meq[2] = rho * (1.0 - 3.0 * v2);
    meq[3] = rho * vx;
    meq[4] = -rho * vx;
    meq[5] = rho * vy;
    meq[6] = -rho * vy;
    meq[7] = rho * (vx * vx - vy * vy);
    meq[8] = rho * vx * vy;
}

/* f_eq = M^-1 m_eq(rho, v). */
void oracle_feq(double rho, double vx, double vy, double* feq) {
    build_mats();
    double meq[Q];
    m_equilibrium(rho, vx, vy, meq);
    for (int a = 0; a < Q; ++a) {
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) acc += Minv[a][k] * meq[k];
        feq[a] = acc;
    }
}

/* ---- collision of one node, Eq. 3, 4, 6, 14 ---------------------------- */

/* Post-collision f* of one node, given its pre-collision f, the force F and
 * the node's psi (the latter only enters Li's term of Eq. 14). g2 = |g|^2,
 * with F = -G psi g, is used only at psi = 0, where |F|^2/psi^2 takes its
 * limit G^2 |g|^2. */
void oracle_collide_node(const oracle_params* P, const double* f, double Fx,
                         double Fy, double psi, double g2, double* fstar) {
    build_mats();
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q; ++a) {
        rho += f[a];
        jx += EX[a] * f[a];
        jy += EY[a] * f[a];
    }
    /* Eq. 6, delta_t = 1 */
    double vx = (jx + 0.5 * Fx) / rho;
    double vy = (jy + 0.5 * Fy) / rho;

    double m[Q], meq[Q], S[Q], mstar[Q];
    for (int k = 0; k < Q; ++k) {
        double acc = 0.0;
        for (int a = 0; a < Q; ++a) acc += Mmat[k][a] * f[a];
        m[k] = acc;
    }
    m_equilibrium(rho, vx, vy, meq);

    /* Eq. 14 */
    double vF = vx * Fx + vy * Fy;
    double F2 = Fx * Fx + Fy * Fy;
    double F2_over_psi2;
    if (psi > 0.0)
        F2_over_psi2 = F2 / (psi * psi);
    else
        F2_over_psi2 = P->G * P->G * g2;
    double tau_e = 1.0 / P->s[1];
    double tau_z = 1.0 / P->s[2];
    S[0] = 0.0;
    S[1] = 6.0 * vF + 0.75 * P->eps * F2_over_psi2 / (tau_e - 0.5);
    S[2] = -6.0 * vF - 0.75 * P->eps * F2_over_psi2 / (tau_z - 0.5);
    S[3] = Fx;
    S[4] = -Fx;
    S[5] = Fy;
    S[6] = -Fy;
    S[7] = 2.0 * (vx * Fx - vy * Fy);
    S[8] = vx * Fy + vy * Fx;

    /* Eq. 3 with delta_t = 1 */
    for (int k = 0; k < Q; ++k)
        mstar[k] = m[k] - P->s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * P->s[k]) * S[k];

    for (int a = 0; a < Q; ++a) {
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) acc += Minv[a][k] * mstar[k];
        fstar[a] = acc;
    }
}

/* ---- initialisation ---------------------------------------------------- */

/* f = f_eq(rho, v) at every node (v = 0 where ux/uy are NULL). */
void oracle_init(const oracle_params* P, const double* rho, const double* ux,
                 const double* uy, double* f) {
    size_t N = (size_t)P->nx * P->ny;
    double feq[Q];
    for (size_t i = 0; i < N; ++i) {
        oracle_feq(rho[i], ux ? ux[i] : 0.0, uy ? uy[i] : 0.0, feq);
        for (int a = 0; a < Q; ++a) f[(size_t)a * N + i] = feq[a];
    }
}

/* ---- one time step ----------------------------------------------------- */

/* Sweep A: rho and psi of every fluid node. */
static unsigned sweep_density_psi(const oracle_params* P, const double* f, double* rho,
                                  double* psi) {
    size_t N = (size_t)P->nx * P->ny;
    unsigned flag = 0;
#pragma omp parallel for num_threads(g_threads) reduction(|:flag) schedule(static)
    for (size_t i = 0; i < N; ++i) {
        int x = (int)(i % P->nx), y = (int)(i / P->nx);
        if (is_solid(P, x, y)) {
            rho[i] = 0.0;
            psi[i] = 0.0;
            continue;
        }
        double r = 0.0;
        for (int a = 0; a < Q; ++a) r += f[(size_t)a * N + i];
        rho[i] = r;
        if (!isfinite(r)) flag |= OR_FLAG_NONFINITE;
        psi[i] = oracle_psi(P, r, &flag);
    }
    return flag;
}

/* Sweep B: force and collision of every fluid node into fstar. */
static void sweep_collide(const oracle_params* P, const double* f, const double* psi,
                          double* fstar) {
    size_t N = (size_t)P->nx * P->ny;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            size_t i = (size_t)y * P->nx + x;
            if (is_solid(P, x, y)) {
                for (int a = 0; a < Q; ++a) fstar[(size_t)a * N + i] = f[(size_t)a * N + i];
                continue;
            }
            double fn[Q], fs[Q];
            double Fx, Fy, g2;
            force_at(P, psi, x, y, &Fx, &Fy, &g2);
            for (int a = 0; a < Q; ++a) fn[a] = f[(size_t)a * N + i];
            oracle_collide_node(P, fn, Fx, Fy, psi[i], g2, fs);
            for (int a = 0; a < Q; ++a) fstar[(size_t)a * N + i] = fs[a];
        }
}

/* Sweep C: Eq. 5 with periodic wrap; a link that would enter a solid node is
 * reflected back into the node it left, as the opposite population. */
static void sweep_stream(const oracle_params* P, const double* fstar, double* f) {
    size_t N = (size_t)P->nx * P->ny;
    /* each f_a(x) of a fluid node is written once: by the fluid node x - e_a
     * streaming into x, or, when x - e_a is solid, by x's own reflection; a
     * solid node writes only its own values */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            size_t i = (size_t)y * P->nx + x;
            if (is_solid(P, x, y)) {
                for (int a = 0; a < Q; ++a) f[(size_t)a * N + i] = fstar[(size_t)a * N + i];
                continue;
            }
            for (int a = 0; a < Q; ++a) {
                int xt = wrap(x + EX[a], P->nx), yt = wrap(y + EY[a], P->ny);
                if (is_solid(P, xt, yt))
                    f[(size_t)OPP[a] * N + i] = fstar[(size_t)a * N + i];
                else
                    f[(size_t)a * N + (size_t)yt * P->nx + xt] = fstar[(size_t)a * N + i];
            }
        }
}

/* Advance f by nsteps time steps. work must hold 9*N + 2*N doubles.
 * Returns the OR of the flags raised during the run. */
unsigned oracle_step(const oracle_params* P, double* f, double* work, int nsteps) {
    size_t N = (size_t)P->nx * P->ny;
    double* fstar = work;
    double* rho = work + (size_t)Q * N;
    double* psi = rho + N;
    unsigned flag = 0;
    for (int t = 0; t < nsteps; ++t) {
        flag |= sweep_density_psi(P, f, rho, psi);
        sweep_collide(P, f, psi, fstar);
        sweep_stream(P, fstar, f);
    }
    return flag;
}

/* ---- diagnostics ------------------------------------------------------- */

/* rho, v (Eq. 6), p (Eq. 10) at every node; solid nodes get zeros. Any output
 * pointer may be NULL. work must hold 2*N doubles. */
unsigned oracle_moments(const oracle_params* P, const double* f, double* work,
                        double* rho_out, double* ux, double* uy, double* p) {
    size_t N = (size_t)P->nx * P->ny;
    double* rho = work;
    double* psi = work + N;
    unsigned flag = sweep_density_psi(P, f, rho, psi);
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            size_t i = (size_t)y * P->nx + x;
            if (is_solid(P, x, y)) {
                if (rho_out) rho_out[i] = 0.0;
                if (ux) ux[i] = 0.0;
                if (uy) uy[i] = 0.0;
                if (p) p[i] = 0.0;
                continue;
            }
            double Fx, Fy, jx = 0.0, jy = 0.0;
            force_at(P, psi, x, y, &Fx, &Fy, NULL);
            for (int a = 0; a < Q; ++a) {
                jx += EX[a] * f[(size_t)a * N + i];
                jy += EY[a] * f[(size_t)a * N + i];
            }
            if (rho_out) rho_out[i] = rho[i];
            if (ux) ux[i] = (jx + 0.5 * Fx) / rho[i];
            if (uy) uy[i] = (jy + 0.5 * Fy) / rho[i];
            if (p) p[i] = oracle_pressure(P, rho[i], psi[i]);
        }
    return flag;
}

/* Total mass sum over fluid nodes of sum_a f_a, summed in node order. */
double oracle_mass(const oracle_params* P, const double* f) {
    size_t N = (size_t)P->nx * P->ny;
    double m = 0.0;
    for (size_t i = 0; i < N; ++i) {
        int x = (int)(i % P->nx), y = (int)(i / P->nx);
        if (is_solid(P, x, y)) continue;
        for (int a = 0; a < Q; ++a) m += f[(size_t)a * N + i];
    }
    return m;
}

/* Total momentum over the fluid nodes: the sums of rho v of Eq. 6,
 * j + F/2 with j = sum_a e_a f_a and F of Eq. 7, summed in node order.
 * work must hold 2*N doubles. Returns the psi flags of the density sweep. */
unsigned oracle_momentum(const oracle_params* P, const double* f, double* work,
                         double* px, double* py) {
    size_t N = (size_t)P->nx * P->ny;
    double* rho = work;
    double* psi = work + N;
    unsigned flag = sweep_density_psi(P, f, rho, psi);
    double sx = 0.0, sy = 0.0;
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            if (is_solid(P, x, y)) continue;
            size_t i = (size_t)y * P->nx + x;
            double Fx, Fy, jx = 0.0, jy = 0.0;
            force_at(P, psi, x, y, &Fx, &Fy, NULL);
            for (int a = 0; a < Q; ++a) {
                jx += EX[a] * f[(size_t)a * N + i];
                jy += EY[a] * f[(size_t)a * N + i];
            }
            sx += jx + 0.5 * Fx;
            sy += jy + 0.5 * Fy;
        }
    *px = sx;
    *py = sy;
    return flag;
}

/*
 * FP64 CPU oracle for the BeatBox monodomain explicit step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py use it.  It shares no code, header, table or constant with
 * the CUDA library in paper_1605_06015_gb300/csrc.
 *
 * Plain, slow C in double precision, single-threaded unless orc_set_threads
 * asks for more: then the two node loops of orc_run (diffusion terms, then
 * updates) are shared among OpenMP threads.  Each node's arithmetic is the
 * same in either case, so results are bit-identical for any thread count;
 * the threads only serve timing on the host cores and long parity runs.
 * Every function follows
 * one passage of the paper (arXiv:1605.06015, "BeatBox - HPC simulation
 * environment ...") and names it:
 *
 *   - diffusion tensor                  Eq. (sigma)
 *   - stencil weights W = Wbar + Wtilde Eq. (Lu) and the weight definitions
 *                                       that follow it (section "Monodomain
 *                                       diffusion and boundary conditions")
 *   - forward Euler                     Eq. (Euler), section "Explicit solvers"
 *   - Rush-Larsen gates                 Eq. (gate), (RL), (RLcoeff), section
 *                                       "Exponential solvers"
 *   - FitzHugh-Nagumo                   Eq. (FHN)
 *   - ZFK / Nagumo                      Eq. (ZFKbidomV), reaction term
 *   - Barkley                           named in section "Cell models" and in
 *                                       script ez.bbs (Table ezscript); the
 *                                       equations are Barkley (1991)
 *   - Beeler-Reuter                     named in section "Cell models"
 *                                       (ionic format); the equations and
 *                                       constants are Beeler & Reuter (1977).
 *                                       The paper does not print them;
 *                                       physics/physiology pins catch gross
 *                                       slips, not small ones: PARITY
 *                                       PARTIAL for the constants' values.
 *   - matrix Rush-Larsen                Eq. (markov-generic) and the scheme
 *                                       u_{n+1} = T(V_n) u_n, T = exp(dt A(V_n))
 *                                       that follows it (section "Exponential
 *                                       solvers"), on the Markov form of the
 *                                       BR sodium activation m^3: a chain of
 *                                       the number k = 0..3 of activated
 *                                       subunits (the paper prints no Markov
 *                                       model).  T is the matrix exponential
 *                                       by its power series (scaling and
 *                                       squaring), not by diagonalisation.
 *   - activation time                   k_poincare device (Appendix, sample.bbs)
 *   - total over tissue                 reduce device (Appendix, sample.bbs)
 *   - idle-partition elision            section "Domain partitioning"
 *
 * Readings of the paper where it is garbled or silent (applied here):
 *   - FHN: u - u^3/3, not u - u^2/3 (the model is the "cubic" fhncub).
 *   - RL: y_{n+1} = A y_n + B (the printed A + B y_n does not keep the fixed
 *     point and contradicts "exact if V = const").
 *   - Eq. (Lu): d_j (D_jk d_k u).
 *   - Wtilde needs D at p +- q_j: where that node is void (or outside the
 *     array) D^p is used in its place.
 *   - Stimulus current is depolarising: dV/dt += +I_stim / Cm.
 *   - Nodes outside the array are void (psi = 0); no ghost rows are stored.
 *   - Activation: first step n+1 with V^n < theta <= V^{n+1}.
 *
 * Layout: dense, x fastest: idx = x + nx*(y + ny*z).  State is SoA in double:
 * state[v*N + idx].  Void nodes are never updated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_FIBRE (-3)
#define ORC_ERR_NOMEM (-8)

enum { ORC_FHN = 1, ORC_BARKLEY = 2, ORC_BR = 3, ORC_ZFK = 4, ORC_DIFFUSION = 5, ORC_BR_MRL = 6, ORC_BR_FCA = 7 };
#define ORC_MAXS 11

typedef struct {
    int nx, ny, nz;
    double h;
    const unsigned char* psi; /* NULL: every node in the array is tissue */
    const float* fib;         /* NULL: isotropic; else 3*N, interleaved x,y,z */
    double Dpar, Dperp;       /* isotropic case uses Dpar */
} orc_geom;

static size_t gidx(const orc_geom* g, int x, int y, int z) {
    return (size_t)x + (size_t)g->nx * ((size_t)y + (size_t)g->ny * (size_t)z);
}

/* Grid indicator function psi_p: 1 inside the tissue, 0 in the void and
 * outside the array. */
static int psi_at(const orc_geom* g, int x, int y, int z) {
    if (x < 0 || y < 0 || z < 0 || x >= g->nx || y >= g->ny || z >= g->nz) return 0;
    if (!g->psi) return 1;
    return g->psi[gidx(g, x, y, z)] != 0;
}

/* Eq. (sigma): D_jk = Dperp delta_jk + (Dpar - Dperp) f_j f_k, f the unit
 * fibre vector.  Returns ORC_ERR_FIBRE for a zero fibre. */
static int tensor_at(const orc_geom* g, size_t idx, double D[3][3]) {
    double f[3] = {0, 0, 0};
    double dpar = g->Dpar, dperp = g->Dperp;
    if (g->fib) {
        double n2 = 0;
        for (int j = 0; j < 3; j++) {
            f[j] = (double)g->fib[3 * idx + j];
            n2 += f[j] * f[j];
        }
        if (!(n2 > 0)) return ORC_ERR_FIBRE;
        double n = sqrt(n2);
        for (int j = 0; j < 3; j++) f[j] /= n;
    } else {
        dperp = dpar; /* isotropic */
    }
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++)
            D[j][k] = (j == k ? dperp : 0.0) + (dpar - dperp) * f[j] * f[k];
    return ORC_OK;
}

int orc_diffusion_tensor(const orc_geom* g, int x, int y, int z, double* D9) {
    double D[3][3];
    int rc = tensor_at(g, gidx(g, x, y, z), D);
    for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++) D9[3 * j + k] = D[j][k];
    return rc;
}

int orc_check_fibres(const orc_geom* g) {
    if (!g->fib) return ORC_OK;
    for (int z = 0; z < g->nz; z++)
        for (int y = 0; y < g->ny; y++)
            for (int x = 0; x < g->nx; x++) {
                if (!psi_at(g, x, y, z)) continue; /* void fibres are ignored */
                double D[3][3];
                if (tensor_at(g, gidx(g, x, y, z), D) != ORC_OK) return ORC_ERR_FIBRE;
            }
    return ORC_OK;
}

/* D at node p + s*q_j, with the reading that a void (or out-of-array)
 * neighbour takes D^p. */
static void tensor_or_centre(const orc_geom* g, int x, int y, int z, int j, int s,
                             const double Dp[3][3], double D[3][3]) {
    int c[3] = {x, y, z};
    c[j] += s;
    if (psi_at(g, c[0], c[1], c[2])) {
        tensor_at(g, gidx(g, c[0], c[1], c[2]), D);
    } else {
        memcpy(D, Dp, sizeof(double) * 9);
    }
}

/* Stencil weights W^p_q = Wbar^p_q + Wtilde^p_q of the section "Monodomain
 * diffusion and boundary conditions", for q in {0,+-1}^3, stored at
 * W[(qx+1) + 3*(qy+1) + 9*(qz+1)].  The centre weight is minus the sum of
 * the others.  The node p must be tissue. */
void orc_cell_weights(const orc_geom* g, int x, int y, int z, double* W) {
    double Dp[3][3];
    tensor_at(g, gidx(g, x, y, z), Dp);
    const double h2 = g->h * g->h;

    /* Wtilde ingredient: S_k = sum_j (D^{p+q_j}_jk - D^{p-q_j}_jk). */
    double S[3] = {0, 0, 0};
    for (int j = 0; j < 3; j++) {
        double Dplus[3][3], Dminus[3][3];
        tensor_or_centre(g, x, y, z, j, +1, Dp, Dplus);
        tensor_or_centre(g, x, y, z, j, -1, Dp, Dminus);
        for (int k = 0; k < 3; k++) S[k] += Dplus[j][k] - Dminus[j][k];
    }

    double sum = 0;
    for (int qz = -1; qz <= 1; qz++)
        for (int qy = -1; qy <= 1; qy++)
            for (int qx = -1; qx <= 1; qx++) {
                int q[3] = {qx, qy, qz};
                int slot = (qx + 1) + 3 * (qy + 1) + 9 * (qz + 1);
                int nnz = (qx != 0) + (qy != 0) + (qz != 0);
                if (nnz == 0) { W[slot] = 0; continue; }
                double psi_q = psi_at(g, x + qx, y + qy, z + qz);
                double wbar = 0, wtil = 0;
                if (nnz == 1) {
                    /* q = +-q_k: Wbar = psi_{p+q} D_kk / h^2, and
                     * Wtilde = +-psi_{p+q} psi_{p-q} S_k / (4 h^2). */
                    int k = qx ? 0 : (qy ? 1 : 2);
                    int s = q[k];
                    double psi_mq = psi_at(g, x - qx, y - qy, z - qz);
                    wbar = psi_q * Dp[k][k] / h2;
                    wtil = (double)s * psi_q * psi_mq * S[k] / (4.0 * h2);
                } else if (nnz == 2) {
                    /* q = +-(q_j + q_k): +D_jk / (2h^2);  q = +-(q_j - q_k):
                     * -D_jk / (2h^2); both times psi_{p+q}. */
                    int j = -1, k = -1;
                    for (int a = 0; a < 3; a++)
                        if (q[a]) { if (j < 0) j = a; else k = a; }
                    double sign = (q[j] * q[k] > 0) ? 1.0 : -1.0;
                    wbar = sign * psi_q * Dp[j][k] / (2.0 * h2);
                } else {
                    wbar = 0; /* corners: 0 */
                }
                W[slot] = wbar + wtil;
                sum += W[slot];
            }
    W[13] = -sum; /* W^p_{(0,0,0)} = - sum_{q != 0} W^p_q */
}

/* (L u)_p = sum_q W^p_q u_{p+q}, written in the equivalent difference form
 * sum_{q != 0} W^p_q (u_{p+q} - u_p), which makes L(const) exactly zero. */
static double apply_weights(const orc_geom* g, const double* W, const double* u,
                            int x, int y, int z) {
    double up = u[gidx(g, x, y, z)];
    double acc = 0;
    for (int qz = -1; qz <= 1; qz++)
        for (int qy = -1; qy <= 1; qy++)
            for (int qx = -1; qx <= 1; qx++) {
                int slot = (qx + 1) + 3 * (qy + 1) + 9 * (qz + 1);
                if (slot == 13 || W[slot] == 0.0) continue;
                acc += W[slot] * (u[gidx(g, x + qx, y + qy, z + qz)] - up);
            }
    return acc;
}

void orc_apply_L(const orc_geom* g, const double* u, double* Lu) {
    double W[27];
    for (int z = 0; z < g->nz; z++)
        for (int y = 0; y < g->ny; y++)
            for (int x = 0; x < g->nx; x++) {
                size_t i = gidx(g, x, y, z);
                if (!psi_at(g, x, y, z)) { Lu[i] = 0; continue; }
                orc_cell_weights(g, x, y, z, W);
                Lu[i] = apply_weights(g, W, u, x, y, z);
            }
}

/* ------------------------------------------------------------------------ */
/* Cell models                                                               */
/* ------------------------------------------------------------------------ */

int orc_nvars(int model) {
    switch (model) {
        case ORC_FHN: return 2;
        case ORC_BARKLEY: return 2;
        case ORC_ZFK: return 1;
        case ORC_BR: return 8;
        case ORC_DIFFUSION: return 1;
        case ORC_BR_MRL: return 11;
        case ORC_BR_FCA: return 11;
    }
    return 0;
}

/* Default parameters; par arrays shorter than these keep the defaults. */
static void model_params(int model, const double* par, int npar, double* p) {
    double d[8] = {0};
    int n = 0;
    switch (model) {
        case ORC_FHN: d[0] = 0.3; d[1] = 0.71; d[2] = 0.5; n = 3; break;   /* eps, beta, gamma */
        case ORC_BARKLEY: d[0] = 0.75; d[1] = 0.02; d[2] = 0.02; n = 3; break; /* a, b, eps */
        case ORC_ZFK: d[0] = 0.13; n = 1; break;                            /* alpha */
        case ORC_BR:
        case ORC_BR_MRL: d[0] = 4.0; d[1] = 0.003; d[2] = 50.0; d[3] = 0.09; n = 4; break;
            /* gNa, gNaC, ENa, gs */
        case ORC_BR_FCA:
            d[0] = 4.0; d[1] = 0.003; d[2] = 50.0; d[3] = 0.09; d[4] = 5e-6; d[5] = 2.0; d[6] = 0.05; d[7] = 0.0;
            n = 8;
            break; /* gNa, gNaC, ENa, gs, Kc (mol/L), tau_c (ms), eps, onfly */
    }
    for (int i = 0; i < 8; i++) p[i] = (i < npar && i < n && par) ? par[i] : d[i];
}

/* Beeler & Reuter (1977) rate constants, in the generic form
 * (C1 exp(C2 (V+C3)) + C4 (V+C5)) / (exp(C6 (V+C3)) + C7); V in mV, rates in
 * 1/ms.  Rows: alpha, beta for x1, m, h, j, d, f.  Transcribed from the
 * primary publication (not printed in the BeatBox paper). */
static const double BR_C[12][7] = {
    /* alpha_x1 */ {0.0005, 0.083, 50.0, 0.0, 0.0, 0.057, 1.0},
    /* beta_x1  */ {0.0013, -0.06, 20.0, 0.0, 0.0, -0.04, 1.0},
    /* alpha_m  */ {0.0, 0.0, 47.0, -1.0, 47.0, -0.1, -1.0},
    /* beta_m   */ {40.0, -0.056, 72.0, 0.0, 0.0, 0.0, 0.0},
    /* alpha_h  */ {0.126, -0.25, 77.0, 0.0, 0.0, 0.0, 0.0},
    /* beta_h   */ {1.7, 0.0, 22.5, 0.0, 0.0, -0.082, 1.0},
    /* alpha_j  */ {0.055, -0.25, 78.0, 0.0, 0.0, -0.2, 1.0},
    /* beta_j   */ {0.3, 0.0, 32.0, 0.0, 0.0, -0.1, 1.0},
    /* alpha_d  */ {0.095, -0.01, -5.0, 0.0, 0.0, -0.072, 1.0},
    /* beta_d   */ {0.07, -0.017, 44.0, 0.0, 0.0, 0.05, 1.0},
    /* alpha_f  */ {0.012, -0.008, 28.0, 0.0, 0.0, 0.15, 1.0},
    /* beta_f   */ {0.0065, -0.02, 30.0, 0.0, 0.0, -0.2, 1.0},
};

static double br_rate(const double* C, double V) {
    double num = C[0] * exp(C[1] * (V + C[2])) + C[3] * (V + C[4]);
    if (C[6] == -1.0) {
        /* exp(z) - 1, with the removable singularity of alpha_m at V = -C3
         * (numerator C4 (V+C5) with C5 = C3 and C1 = 0) taken as its limit. */
        double z = C[5] * (V + C[2]);
        if (z == 0.0 && C[0] == 0.0 && C[4] == C[2]) return C[3] / C[5];
        return num / expm1(z);
    }
    return num / (exp(C[5] * (V + C[2])) + C[6]);
}

/* State order for BR: V, Ca, x1, m, h, j, d, f. */
enum { BR_V = 0, BR_CA, BR_X1, BR_M, BR_H, BR_J, BR_D, BR_F };

void orc_br_rates(double V, double* alpha6, double* beta6) {
    for (int g = 0; g < 6; g++) {
        alpha6[g] = br_rate(BR_C[2 * g], V);
        beta6[g] = br_rate(BR_C[2 * g + 1], V);
    }
}

/* BR (1977) membrane currents in uA/cm^2 and dCa/dt, with the open
 * probability m3 of the sodium activation given.  out[0] = I_ion,
 * out[1] = I_s, out[2] = dCa/dt. */
static void br_currents_m3(const double* p, double V, double Ca, double x1, double m3, double hh, double j,
                           double d, double f, double* out) {
    double gNa = p[0], gNaC = p[1], ENa = p[2], gs = p[3];
    double INa = (gNa * m3 * hh * j + gNaC) * (V - ENa);
    double Es = -82.3 - 13.0287 * log(Ca);
    double Is = gs * d * f * (V - Es);
    double Ix1 = x1 * 0.8 * (exp(0.04 * (V + 77.0)) - 1.0) / exp(0.04 * (V + 35.0));
    double w = V + 23.0;
    double lin = (w == 0.0) ? 0.2 / 0.04 : 0.2 * w / (-expm1(-0.04 * w));
    double IK1 = 0.35 * (4.0 * (exp(0.04 * (V + 85.0)) - 1.0) /
                             (exp(0.08 * (V + 53.0)) + exp(0.04 * (V + 53.0))) +
                         lin);
    out[0] = INa + Is + Ix1 + IK1;
    out[1] = Is;
    out[2] = -1e-7 * Is + 0.07 * (1e-7 - Ca);
}

void orc_br_currents(const double* p, const double* y, double* out) {
    double m = y[BR_M];
    br_currents_m3(p, y[BR_V], y[BR_CA], y[BR_X1], m * m * m, y[BR_H], y[BR_J], y[BR_D], y[BR_F], out);
}

/* ---- Markov form of the BR sodium activation (matrix Rush-Larsen) ------- */

/* State order of the Markov variant: V, Ca, x1, h, j, d, f, then P0..P3, the
 * probabilities that k = 0..3 of the three activation subunits are open
 * (P3 takes the place of m^3). */
enum { MR_V = 0, MR_CA, MR_X1, MR_H, MR_J, MR_D, MR_F, MR_P0 };

/* Transition-rate matrix of Eq. (markov-generic), du/dt = A u, for the
 * chain: k -> k+1 at (3-k) alpha_m, k -> k-1 at k beta_m.  Row-major,
 * A[i][j] = rate from state j into state i (columns sum to zero). */
void orc_mrl_generator(double V, double* A16) {
    double al[6], be[6];
    orc_br_rates(V, al, be);
    const double a = al[1], b = be[1]; /* alpha_m, beta_m */
    for (int i = 0; i < 16; i++) A16[i] = 0.0;
    for (int k = 0; k < 4; k++) {
        double out = 0.0;
        if (k < 3) { A16[(k + 1) * 4 + k] = (3 - k) * a; out += (3 - k) * a; }
        if (k > 0) { A16[(k - 1) * 4 + k] = k * b; out += k * b; }
        A16[k * 4 + k] = -out;
    }
}

static void mat4_mul(const double* X, const double* Y, double* Z) {
    double t[16];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            double s = 0.0;
            for (int k = 0; k < 4; k++) s += X[i * 4 + k] * Y[k * 4 + j];
            t[i * 4 + j] = s;
        }
    memcpy(Z, t, sizeof(t));
}

static void mat4_expm(const double* A16, double dt, double* T16);

/* T = exp(dt A(V)) of the scheme u_{n+1} = T(V_n) u_n (mat4_expm below). */

void orc_mrl_transition(double V, double dt, double* T16) {
    double M[16];
    orc_mrl_generator(V, M);
    mat4_expm(M, dt, T16);
}

/* exp(dt A) for a 4 x 4 matrix A: the power series sum_k M^k / k! of M = dt A
 * / 2^s (s chosen so that the largest absolute row sum of M is at most 1/2; 30
 * terms), squared s times. */
static void mat4_expm(const double* A16, double dt, double* T16) {
    double M[16];
    memcpy(M, A16, sizeof(M));
    double nrm = 0.0;
    for (int i = 0; i < 4; i++) {
        double r = 0.0;
        for (int j = 0; j < 4; j++) r += fabs(M[i * 4 + j]) * dt;
        if (r > nrm) nrm = r;
    }
    int s = 0;
    while (nrm > 0.5) { nrm *= 0.5; s++; }
    const double sc = dt / ldexp(1.0, s);
    for (int i = 0; i < 16; i++) M[i] *= sc;
    double term[16], E[16];
    for (int i = 0; i < 16; i++) term[i] = E[i] = (i % 5 == 0) ? 1.0 : 0.0;
    for (int k = 1; k <= 30; k++) {
        mat4_mul(term, M, term);
        for (int i = 0; i < 16; i++) term[i] /= k;
        for (int i = 0; i < 16; i++) E[i] += term[i];
    }
    for (int q = 0; q < s; q++) mat4_mul(E, E, E);
    memcpy(T16, E, sizeof(E));
}

/* ---- a Markov chain with two control variables (multivariate matrix RL) --- */

/* Beeler-Reuter with the inactivation of the slow inward current as a
 * two-gate channel: the voltage-dependent gate f of the 1977 model (rates
 * alpha_f, beta_f) and a calcium-dependent gate c, closed -> open at
 * alpha_c = c_inf / tau_c, open -> closed at beta_c = (1 - c_inf) / tau_c,
 * c_inf = 1 / (1 + Ca / Kc).  The channel's four states q = f + 2 c (f, c in
 * {0, 1}: gate open) obey Eq. (markov-generic) with A(V, Ca) = A_f(V) (+)
 * A_c(Ca) + R(V, Ca): the Kronecker sum of the two gates' univariate
 * generators plus a small multivariate remainder, a direct transition from
 * (f open, c closed) to (f closed, c open) at rate eps alpha_f(V) (1 -
 * c_inf(Ca)).  I_s = g_s d Q3 (V - E_s), Q3 = P(f and c open).  The paper
 * prints no such model; it exercises the scheme of section "Exponential
 * solvers" for a matrix depending on V and Ca: Lie splitting into the
 * univariate subsystems, each advanced by its exact (matrix Rush-Larsen)
 * step, and forward Euler for the remainder.  State order: V, Ca, x1, m, h,
 * j, d, Q0, Q1, Q2, Q3. */
enum { FC_V = 0, FC_CA, FC_X1, FC_M, FC_H, FC_J, FC_D, FC_Q0 };

static double fca_cinf(const double* p, double Ca) { return 1.0 / (1.0 + Ca / p[4]); }

/* The generator A(V, Ca) of the channel (row-major, A[i][j] = rate from
 * state j into state i; columns sum to zero). */
void orc_fca_generator(const double* par, int npar, double V, double Ca, double* A16) {
    double p[8], al[6], be[6];
    model_params(ORC_BR_FCA, par, npar, p);
    orc_br_rates(V, al, be);
    const double af = al[5], bf = be[5], ci = fca_cinf(p, Ca);
    const double ac = ci / p[5], bc = (1.0 - ci) / p[5], r = p[6] * af * (1.0 - ci);
    for (int i = 0; i < 16; i++) A16[i] = 0.0;
    for (int q = 0; q < 4; q++) {
        const int f = q & 1, c = q >> 1;
        const int qf = q ^ 1, qc = q ^ 2;  /* the states one gate away */
        A16[qf * 4 + q] += f ? bf : af;
        A16[qc * 4 + q] += c ? bc : ac;
    }
    A16[2 * 4 + 1] += r; /* (f open, c closed) -> (f closed, c open) */
    for (int q = 0; q < 4; q++) {
        double out = 0.0;
        for (int i = 0; i < 4; i++)
            if (i != q) out += A16[i * 4 + q];
        A16[q * 4 + q] = -out;
    }
}

/* The exact step of a two-state gate with rates a (closed -> open) and b
 * (open -> closed) applied to one index of the channel's state: Eq. (RL)
 * for the open probability, A = exp(-(a+b) dt), B = a/(a+b) (1 - A), as the
 * 2 x 2 transition matrix [[1-B, 1-A-B], [B, A+B]] (columns: from closed,
 * from open), on the pairs of states that differ in the gate `bit`. */
static void gate2_step(double a, double b, double dt, int bit, double* u) {
    const double A = exp(-(a + b) * dt), B = a / (a + b) * (1.0 - A);
    for (int q = 0; q < 4; q++) {
        if (q & bit) continue;
        const double u0 = u[q], u1 = u[q | bit];
        u[q] = (1.0 - B) * u0 + (1.0 - A - B) * u1;
        u[q | bit] = B * u0 + (A + B) * u1;
    }
}

/* The multivariate matrix Rush-Larsen step of the channel with V and Ca held
 * at their values at the start of the step: the voltage gate's exact step,
 * then the calcium gate's, then forward Euler for the remainder R. */
void orc_fca_split_step(const double* par, int npar, double V, double Ca, double dt, const double* u, double* un) {
    double p[8], al[6], be[6], w[4];
    model_params(ORC_BR_FCA, par, npar, p);
    orc_br_rates(V, al, be);
    const double ci = fca_cinf(p, Ca);
    for (int q = 0; q < 4; q++) w[q] = u[q];
    gate2_step(al[5], be[5], dt, 1, w);
    gate2_step(ci / p[5], (1.0 - ci) / p[5], dt, 2, w);
    const double r = p[6] * al[5] * (1.0 - ci);
    for (int q = 0; q < 4; q++) un[q] = w[q];
    un[1] -= dt * r * w[1];
    un[2] += dt * r * w[1];
}

/* The same step without splitting: u_{n+1} = exp(dt A(V, Ca)) u_n, the matrix
 * exponential of the whole generator (the "on the fly" matrix Rush-Larsen). */
void orc_fca_exact_step(const double* par, int npar, double V, double Ca, double dt, const double* u, double* un) {
    double A[16], T[16];
    orc_fca_generator(par, npar, V, Ca, A);
    mat4_expm(A, dt, T);
    for (int i = 0; i < 4; i++) {
        double s = 0.0;
        for (int j = 0; j < 4; j++) s += T[i * 4 + j] * u[j];
        un[i] = s;
    }
}

/* One unsplit step of one node: Eq. (Euler) for the non-gate variables with
 * the diffusion term L and the stimulus added to the voltage equation, and
 * Eq. (RL) (read as y' = A y + B) for the BR gates. */
void orc_cell_update(int model, const double* par, int npar, const double* y, double L,
                     double Istim, double dt, double* yn) {
    double p[8];
    model_params(model, par, npar, p);
    switch (model) {
        case ORC_FHN: {
            double u = y[0], v = y[1], eps = p[0], bet = p[1], gam = p[2];
            yn[0] = u + dt * ((u - u * u * u / 3.0 - v) / eps + L + Istim);
            yn[1] = v + dt * (eps * (u + bet - gam * v));
        } break;
        case ORC_BARKLEY: {
            double u = y[0], v = y[1], a = p[0], b = p[1], eps = p[2];
            yn[0] = u + dt * (u * (1.0 - u) * (u - (v + b) / a) / eps + L + Istim);
            yn[1] = v + dt * (u - v);
        } break;
        case ORC_ZFK: {
            double u = y[0], alpha = p[0];
            yn[0] = u + dt * (u * (u - alpha) * (1.0 - u) + L + Istim);
        } break;
        case ORC_DIFFUSION: {
            /* no reaction: the diffusion equation alone (used by the
             * section's J0 disc test) */
            yn[0] = y[0] + dt * (L + Istim);
        } break;
        case ORC_BR: {
            const double Cm = 1.0;
            double cur[3], al[6], be[6];
            orc_br_currents(p, y, cur);
            orc_br_rates(y[BR_V], al, be);
            yn[BR_V] = y[BR_V] + dt * (-(cur[0] - Istim) / Cm + L);
            yn[BR_CA] = y[BR_CA] + dt * cur[2];
            for (int g = 0; g < 6; g++) {
                double A = exp(-(al[g] + be[g]) * dt);
                double B = al[g] / (al[g] + be[g]) * (1.0 - A);
                yn[BR_X1 + g] = A * y[BR_X1 + g] + B;
            }
        } break;
        case ORC_BR_MRL: {
            /* as ORC_BR, with m^3 = P3 and the chain advanced by matrix
             * Rush-Larsen; the gates x1, h, j, d, f by Eq. (RL) */
            const double Cm = 1.0;
            double cur[3], al[6], be[6], T[16];
            br_currents_m3(p, y[MR_V], y[MR_CA], y[MR_X1], y[MR_P0 + 3], y[MR_H], y[MR_J], y[MR_D], y[MR_F], cur);
            orc_br_rates(y[MR_V], al, be);
            yn[MR_V] = y[MR_V] + dt * (-(cur[0] - Istim) / Cm + L);
            yn[MR_CA] = y[MR_CA] + dt * cur[2];
            const int gate_of[5] = {0, 2, 3, 4, 5}; /* x1, h, j, d, f in the rate table */
            for (int q = 0; q < 5; q++) {
                const int g = gate_of[q];
                double A = exp(-(al[g] + be[g]) * dt);
                double B = al[g] / (al[g] + be[g]) * (1.0 - A);
                yn[MR_X1 + q] = A * y[MR_X1 + q] + B;
            }
            orc_mrl_transition(y[MR_V], dt, T);
            for (int i = 0; i < 4; i++) {
                double s = 0.0;
                for (int j = 0; j < 4; j++) s += T[i * 4 + j] * y[MR_P0 + j];
                yn[MR_P0 + i] = s;
            }
        } break;
        case ORC_BR_FCA: {
            /* Eq. (Euler) for V and Ca with I_s = g_s d Q3 (V - E_s), Eq.
             * (RL) for x1, m, h, j, d, and the channel by the split matrix
             * Rush-Larsen step at (V, Ca) of the start of the step, or with
             * the parameter onfly set by the unsplit exponential */
            const double Cm = 1.0;
            double cur[3], al[6], be[6];
            const double m = y[FC_M];
            br_currents_m3(p, y[FC_V], y[FC_CA], y[FC_X1], m * m * m, y[FC_H], y[FC_J], y[FC_D], y[FC_Q0 + 3], cur);
            orc_br_rates(y[FC_V], al, be);
            yn[FC_V] = y[FC_V] + dt * (-(cur[0] - Istim) / Cm + L);
            yn[FC_CA] = y[FC_CA] + dt * cur[2];
            for (int g = 0; g < 5; g++) { /* x1, m, h, j, d: the first five rates */
                double A = exp(-(al[g] + be[g]) * dt);
                double B = al[g] / (al[g] + be[g]) * (1.0 - A);
                yn[FC_X1 + g] = A * y[FC_X1 + g] + B;
            }
            if (p[7] != 0.0) /* onfly: the unsplit exponential of the whole generator */
                orc_fca_exact_step(par, npar, y[FC_V], y[FC_CA], dt, y + FC_Q0, yn + FC_Q0);
            else
                orc_fca_split_step(par, npar, y[FC_V], y[FC_CA], dt, y + FC_Q0, yn + FC_Q0);
        } break;
    }
}

/* Right-hand side of the ODE form of a model (section "Explicit solvers",
 * Eq. (ODE)) with the diffusion term and stimulus together as a source I held
 * fixed over the step on the voltage equation.  Models given by a right-hand
 * side only (FHN, Barkley, ZFK, diffusion); returns ORC_ERR_ARG otherwise. */
static int model_rhs(int model, const double* p, const double* y, double I, double* dy) {
    switch (model) {
        case ORC_FHN:
            dy[0] = (y[0] - y[0] * y[0] * y[0] / 3.0 - y[1]) / p[0] + I;
            dy[1] = p[0] * (y[0] + p[1] - p[2] * y[1]);
            return ORC_OK;
        case ORC_BARKLEY:
            dy[0] = y[0] * (1.0 - y[0]) * (y[0] - (y[1] + p[1]) / p[0]) / p[2] + I;
            dy[1] = y[0] - y[1];
            return ORC_OK;
        case ORC_ZFK:
            dy[0] = y[0] * (y[0] - p[0]) * (1.0 - y[0]) + I;
            return ORC_OK;
        case ORC_DIFFUSION:
            dy[0] = I;
            return ORC_OK;
    }
    return ORC_ERR_ARG;
}

/* One step of the classical fourth-order Runge-Kutta scheme (the rk4
 * kinetics solver of section "Explicit solvers") for the ODE of model_rhs with
 * the source L + Istim: stages at t, t + dt/2, t + dt/2 and t + dt, weights
 * 1/6, 1/3, 1/3, 1/6. */
int orc_cell_update_rk4(int model, const double* par, int npar, const double* y, double L, double Istim,
                        double dt, double* yn) {
    double p[8], k1[ORC_MAXS], k2[ORC_MAXS], k3[ORC_MAXS], k4[ORC_MAXS], t[ORC_MAXS];
    model_params(model, par, npar, p);
    const int S = orc_nvars(model);
    const double I = L + Istim;
    if (model_rhs(model, p, y, I, k1)) return ORC_ERR_ARG;
    for (int v = 0; v < S; v++) t[v] = y[v] + 0.5 * dt * k1[v];
    model_rhs(model, p, t, I, k2);
    for (int v = 0; v < S; v++) t[v] = y[v] + 0.5 * dt * k2[v];
    model_rhs(model, p, t, I, k3);
    for (int v = 0; v < S; v++) t[v] = y[v] + dt * k3[v];
    model_rhs(model, p, t, I, k4);
    for (int v = 0; v < S; v++) yn[v] = y[v] + dt / 6.0 * (k1[v] + 2.0 * k2[v] + 2.0 * k3[v] + k4[v]);
    return ORC_OK;
}

/* Rest state of a model: FHN by Newton on the cubic, Barkley and ZFK at 0,
 * BR by integrating the space-clamped cell (dt = 0.01 ms) for 20 s. */
int orc_rest_state(int model, const double* par, int npar, double* y) {
    double p[8];
    model_params(model, par, npar, p);
    switch (model) {
        case ORC_FHN: {
            /* v = (u + beta)/gamma, u - u^3/3 - v = 0. */
            double u = -1.0;
            for (int it = 0; it < 100; it++) {
                double F = u - u * u * u / 3.0 - (u + p[1]) / p[2];
                double dF = 1.0 - u * u - 1.0 / p[2];
                u -= F / dF;
            }
            y[0] = u;
            y[1] = (u + p[1]) / p[2];
        } return ORC_OK;
        case ORC_BARKLEY: y[0] = 0; y[1] = 0; return ORC_OK;
        case ORC_ZFK: y[0] = 0; return ORC_OK;
        case ORC_DIFFUSION: y[0] = 0; return ORC_OK;
        case ORC_BR: {
            double al[6], be[6], yn[8];
            y[BR_V] = -84.0;
            y[BR_CA] = 1e-7;
            orc_br_rates(y[BR_V], al, be);
            for (int g = 0; g < 6; g++) y[BR_X1 + g] = al[g] / (al[g] + be[g]);
            for (int n = 0; n < 2000000; n++) {
                orc_cell_update(model, par, npar, y, 0.0, 0.0, 0.01, yn);
                memcpy(y, yn, sizeof(double) * 8);
            }
        } return ORC_OK;
        case ORC_BR_MRL: {
            /* the BR rest state with the chain at the binomial distribution
             * of m (independent subunits) */
            double r[8];
            orc_rest_state(ORC_BR, par, npar, r);
            const double m = r[BR_M];
            y[MR_V] = r[BR_V]; y[MR_CA] = r[BR_CA]; y[MR_X1] = r[BR_X1];
            y[MR_H] = r[BR_H]; y[MR_J] = r[BR_J]; y[MR_D] = r[BR_D]; y[MR_F] = r[BR_F];
            y[MR_P0 + 0] = (1 - m) * (1 - m) * (1 - m);
            y[MR_P0 + 1] = 3 * m * (1 - m) * (1 - m);
            y[MR_P0 + 2] = 3 * m * m * (1 - m);
            y[MR_P0 + 3] = m * m * m;
        } return ORC_OK;
        case ORC_BR_FCA: {
            /* from the BR rest state with the channel at the product of the
             * two gates' steady states, the space-clamped cell integrated
             * for 20 s at dt = 0.01 ms (the calcium gate moves the rest) */
            double r[8], yn[ORC_MAXS];
            orc_rest_state(ORC_BR, par, npar, r);
            for (int v = 0; v < 7; v++) y[v] = r[v]; /* V, Ca, x1, m, h, j, d share the BR order */
            const double f = r[BR_F], c = fca_cinf(p, r[BR_CA]);
            y[FC_Q0 + 0] = (1 - f) * (1 - c);
            y[FC_Q0 + 1] = f * (1 - c);
            y[FC_Q0 + 2] = (1 - f) * c;
            y[FC_Q0 + 3] = f * c;
            for (int n = 0; n < 2000000; n++) {
                orc_cell_update(model, par, npar, y, 0.0, 0.0, 0.01, yn);
                memcpy(y, yn, sizeof(double) * 11);
            }
        } return ORC_OK;
    }
    return ORC_ERR_ARG;
}

/* ------------------------------------------------------------------------ */
/* Whole-grid time stepping                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int model;
    const double* par;
    int npar;
    const unsigned char* stim; /* NULL: no stimulus region */
    double amp, t_on, t_off;
    double theta;
    int split; /* 0: unsplit (diff + euler); 1: Lie splitting (diffstep, then the kinetics step) */
    int rk4;   /* kinetics solver: 0 forward Euler (Rush-Larsen gates for BR), 1 classical RK4 (rhs models) */
} orc_run_cfg;

static void kinetics(const orc_run_cfg* c, const double* y, double L, double Is, double dt, double* yn) {
    if (c->rk4)
        orc_cell_update_rk4(c->model, c->par, c->npar, y, L, Is, dt, yn);
    else
        orc_cell_update(c->model, c->par, c->npar, y, L, Is, dt, yn);
}

/* The update of one tissue node from its state y, its diffusion term L and
 * stimulus Is, under the run's scheme.  Unsplit (section "Computation of
 * intermediate expressions"): L enters the voltage equation of the kinetics
 * step.  Lie splitting (section "Operator splitting"): first the diffusion
 * substep V_{n+1/2} = V_n + dt L on its own, then the kinetics step from
 * (V_{n+1/2}, the other variables at n) with no diffusion term; the stimulus
 * belongs to the kinetics step. */
static void node_update(const orc_run_cfg* c, const double* y, double L, double Is, double dt, double* yn) {
    if (!c->split) {
        kinetics(c, y, L, Is, dt, yn);
        return;
    }
    double yh[ORC_MAXS];
    const int S = orc_nvars(c->model);
    for (int v = 0; v < S; v++) yh[v] = y[v];
    yh[0] = y[0] + dt * L;
    kinetics(c, yh, 0.0, Is, dt, yn);
}

/* n_steps unsplit steps (section "Computation of intermediate expressions":
 * diff + euler/rushlarsen) in place on state (SoA, nvars*N doubles).
 * t, n: time and step counter, updated.  act: activation steps (INT32_MAX =
 * not yet), may be NULL.  The weights are built once per call (they depend
 * only on geometry), then every step first evaluates L on all tissue nodes
 * from the old state and then updates every tissue node. */
static int orc_threads = 1;

/* Threads for the node loops of orc_run (1 = serial, the default); returns
 * the count in use (1 when the oracle was built without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
    orc_threads = n < 1 ? 1 : n;
#else
    (void)n;
    orc_threads = 1;
#endif
    return orc_threads;
}

int orc_run(const orc_geom* g, const orc_run_cfg* c, double* state, double dt, int n_steps,
            double* t, long long* n, int32_t* act) {
    const size_t N = (size_t)g->nx * g->ny * g->nz;
    const int S = orc_nvars(c->model);
    if (S == 0 || (c->rk4 && (c->model == ORC_BR || c->model == ORC_BR_MRL || c->model == ORC_BR_FCA))) return ORC_ERR_ARG;
    int rc = orc_check_fibres(g);
    if (rc) return rc;
    size_t nt = 0;
    for (int z = 0; z < g->nz; z++)
        for (int y = 0; y < g->ny; y++)
            for (int x = 0; x < g->nx; x++) nt += psi_at(g, x, y, z);
    int* cx = malloc(sizeof(int) * 3 * (nt ? nt : 1));
    double* W = malloc(sizeof(double) * 27 * (nt ? nt : 1));
    double* L = malloc(sizeof(double) * (nt ? nt : 1));
    if (!cx || !W || !L) { free(cx); free(W); free(L); return ORC_ERR_NOMEM; }
    size_t m = 0;
    for (int z = 0; z < g->nz; z++)
        for (int y = 0; y < g->ny; y++)
            for (int x = 0; x < g->nx; x++)
                if (psi_at(g, x, y, z)) {
                    cx[3 * m] = x; cx[3 * m + 1] = y; cx[3 * m + 2] = z;
                    m++;
                }
    const int nth = orc_threads;
    const long long ntl = (long long)nt;
    (void)nth;
#pragma omp parallel for schedule(static) num_threads(nth) if (nth > 1)
    for (long long i = 0; i < ntl; i++) orc_cell_weights(g, cx[3 * i], cx[3 * i + 1], cx[3 * i + 2], W + 27 * i);
    for (int s = 0; s < n_steps; s++) {
        int on = c->amp != 0.0 && *t >= c->t_on && *t < c->t_off;
        /* every diffusion term from the old state first ... */
#pragma omp parallel for schedule(static) num_threads(nth) if (nth > 1)
        for (long long i = 0; i < ntl; i++)
            L[i] = apply_weights(g, W + 27 * i, state, cx[3 * i], cx[3 * i + 1], cx[3 * i + 2]);
        /* ... then every node's update, each touching only its own node */
#pragma omp parallel for schedule(static) num_threads(nth) if (nth > 1)
        for (long long i = 0; i < ntl; i++) {
            double y[ORC_MAXS], yn[ORC_MAXS];
            size_t p = gidx(g, cx[3 * i], cx[3 * i + 1], cx[3 * i + 2]);
            for (int v = 0; v < S; v++) y[v] = state[(size_t)v * N + p];
            double Is = (on && c->stim && c->stim[p]) ? c->amp : 0.0;
            node_update(c, y, L[i], Is, dt, yn);
            for (int v = 0; v < S; v++) state[(size_t)v * N + p] = yn[v];
            if (act && act[p] == INT32_MAX && y[0] < c->theta && c->theta <= yn[0])
                act[p] = (int32_t)(*n + 1);
        }
        *t += dt;
        *n += 1;
    }
    free(cx); free(W); free(L);
    return ORC_OK;
}

/* One step evaluated only at the listed nodes (linear indices), from a given
 * state, for sampled comparisons on grids too large to step whole.  out is
 * ncells*nvars, node-major.  Void nodes return their input unchanged. */
int orc_step_cells(const orc_geom* g, const orc_run_cfg* c, const double* state, double dt,
                   double t, const long long* cells, int ncells, double* out) {
    const size_t N = (size_t)g->nx * g->ny * g->nz;
    const int S = orc_nvars(c->model);
    if (S == 0 || (c->rk4 && (c->model == ORC_BR || c->model == ORC_BR_MRL || c->model == ORC_BR_FCA))) return ORC_ERR_ARG;
    int on = c->amp != 0.0 && t >= c->t_on && t < c->t_off;
    double W[27], y[ORC_MAXS], yn[ORC_MAXS];
    for (int i = 0; i < ncells; i++) {
        long long p = cells[i];
        int x = (int)(p % g->nx), yy = (int)((p / g->nx) % g->ny), z = (int)(p / ((long long)g->nx * g->ny));
        for (int v = 0; v < S; v++) y[v] = state[(size_t)v * N + p];
        if (!psi_at(g, x, yy, z)) {
            for (int v = 0; v < S; v++) out[(size_t)i * S + v] = y[v];
            continue;
        }
        double Dp[3][3];
        if (tensor_at(g, (size_t)p, Dp) != ORC_OK) return ORC_ERR_FIBRE;
        orc_cell_weights(g, x, yy, z, W);
        double Lp = apply_weights(g, W, state, x, yy, z);
        double Is = (on && c->stim && c->stim[p]) ? c->amp : 0.0;
        node_update(c, y, Lp, Is, dt, yn);
        for (int v = 0; v < S; v++) out[(size_t)i * S + v] = yn[v];
    }
    return ORC_OK;
}

/* reduce device: sum over tissue nodes of a field, in double. */
double orc_total(const orc_geom* g, const double* u) {
    double s = 0;
    for (int z = 0; z < g->nz; z++)
        for (int y = 0; y < g->ny; y++)
            for (int x = 0; x < g->nx; x++)
                if (psi_at(g, x, y, z)) s += u[gidx(g, x, y, z)];
    return s;
}

/* Idle-partition elision inside one grid: the bricks of tx*ty*tz nodes
 * (bricks at the high edges are cut by the array) that hold at least one
 * tissue node, as brick ids bx + nbx*(by + nby*bz) in increasing order, found
 * by visiting every node of every brick.  Returns the count, or -1 if cap is
 * too small. */
long long orc_active_bricks(const orc_geom* g, int tx, int ty, int tz, int32_t* out, long long cap) {
    int nbx = (g->nx + tx - 1) / tx, nby = (g->ny + ty - 1) / ty, nbz = (g->nz + tz - 1) / tz;
    long long cnt = 0;
    for (int bz = 0; bz < nbz; bz++)
        for (int by = 0; by < nby; by++)
            for (int bx = 0; bx < nbx; bx++) {
                int any = 0;
                for (int z = bz * tz; z < (bz + 1) * tz && !any; z++)
                    for (int y = by * ty; y < (by + 1) * ty && !any; y++)
                        for (int x = bx * tx; x < (bx + 1) * tx && !any; x++)
                            any = psi_at(g, x, y, z);
                if (any) {
                    if (cnt >= cap) return -1;
                    out[cnt++] = bx + nbx * (by + nby * bz);
                }
            }
    return cnt;
}

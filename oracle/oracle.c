/*
 * CPU oracle for the QAOA / AQA state-vector path (arXiv 2104.03293).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * reference that the CUDA path is checked against.  It shares no code with
 * the CUDA library (no headers, no helpers, no tables) and nothing in the
 * product path may call it: only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load it.
 *
 * Everything is complex128 / float64 and follows the paper's definitions
 * gate by gate, without any fusion or blocking:
 *
 *   - state vector: 2^n amplitudes psi_{q_{n-1}...q_0}; qubit j is bit j of
 *     the basis index, q_0 the least significant bit (Sec. II.A, the rank-N
 *     tensor written after Eq. (1)).
 *   - single-qubit gates are 2-component updates over all pairs of
 *     amplitudes that differ in bit j (Eq. twocomponentupdates).
 *   - H_C = sum_i h_i Z_i + sum_{i<j} J_ij Z_i Z_j (Eq. HC), diagonal; with
 *     the textbook convention Z|0> = +|0>, i.e. s_i(z) = 1 - 2 bit_i(z).
 *   - H_D = sum_i X_i (Sec. III.A.2, the mixer below Eq. QAOA_state).
 *   - |beta,gamma> = prod_{k=1}^p e^{-i beta_k H_D} e^{-i gamma_k H_C} |+>^n
 *     (Eq. QAOA_state; Appendix A spells out the factor order: the phase of
 *     layer k acts before its mixer).  e^{-i gamma H_C} is applied as one
 *     z-rotation per field term and one ZZ phase per coupling, and
 *     e^{-i beta H_D} as one x-rotation per qubit (Sec. III.B.1, the
 *     paragraph on how JUQCS-G computes the exponentials).
 *   - readout: E = <H_C> and the ground-state ("success") probability, the
 *     total weight on all basis states of minimal cost (Sec. III.B.1 and the
 *     success-probability definition in Sec. III.A.3).
 *
 * The adjoint (reverse-mode derivative of the readout with respect to the
 * 2p angles) is not in the paper.  Here it is the textbook gate-by-gate
 * reverse pass: for every gate G = exp(-i theta A) in reverse order,
 * dF/dtheta = 2 Im <lambda|A|psi> with psi and lambda the states just after
 * that gate, then both are multiplied by G^dagger.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* spin value s_i(z) = 1 - 2 * bit_i(z)  (Z|0> = +|0>) */
static inline double spin(uint64_t z, int i) { return ((z >> i) & 1u) ? -1.0 : 1.0; }

/* Eq. (HC) evaluated on basis state z. */
double orc_cost(int n, const double* h, int m, const int32_t* edges, const double* J, uint64_t z)
{
    double c = 0.0;
    for (int i = 0; i < n; ++i) c += h[i] * spin(z, i);
    for (int e = 0; e < m; ++e) c += J[e] * spin(z, edges[2 * e]) * spin(z, edges[2 * e + 1]);
    return c;
}

/* All 2^n costs (small n only: tests). */
void orc_cost_all(int n, const double* h, int m, const int32_t* edges, const double* J, double* out)
{
    uint64_t N = (uint64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) out[z] = orc_cost(n, h, m, edges, J, (uint64_t)z);
}

/* Ground state by full enumeration (the t_FE search of Table III):
 * minimum and maximum cost, lowest index of a minimiser, number of minimisers. */
void orc_ground(int n, const double* h, int m, const int32_t* edges, const double* J,
                double* cmin_out, double* cmax_out, int64_t* argmin_out, int64_t* count_out)
{
    uint64_t N = (uint64_t)1 << n;
    double cmin = INFINITY, cmax = -INFINITY;
    int64_t argmin = -1, count = 0;
#pragma omp parallel
    {
        double lmin = INFINITY, lmax = -INFINITY;
        int64_t larg = -1, lcnt = 0;
#pragma omp for schedule(static)
        for (int64_t z = 0; z < (int64_t)N; ++z) {
            double c = orc_cost(n, h, m, edges, J, (uint64_t)z);
            if (c < lmin) { lmin = c; larg = z; lcnt = 1; }
            else if (c == lmin) { lcnt++; if (z < larg) larg = z; }
            if (c > lmax) lmax = c;
        }
#pragma omp critical
        {
            if (lmin < cmin) { cmin = lmin; argmin = larg; count = lcnt; }
            else if (lmin == cmin) { count += lcnt; if (larg < argmin) argmin = larg; }
            if (lmax > cmax) cmax = lmax;
        }
    }
    *cmin_out = cmin; *cmax_out = cmax; *argmin_out = argmin; *count_out = count;
}

/* |+>^n : every amplitude 2^{-n/2}. */
void orc_init_plus(int n, cplx* psi)
{
    uint64_t N = (uint64_t)1 << n;
    double a = pow(2.0, -0.5 * n);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) psi[z] = a;
}

/* exp(-i theta Z_i): multiply psi_z by exp(-i theta s_i(z)). */
void orc_gate_z(int n, cplx* psi, int i, double theta)
{
    uint64_t N = (uint64_t)1 << n;
    cplx f0 = cexp(-I * theta), f1 = cexp(I * theta);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) psi[z] *= ((z >> i) & 1) ? f1 : f0;
}

/* exp(-i theta Z_i Z_j): multiply psi_z by exp(-i theta s_i(z) s_j(z)). */
void orc_gate_zz(int n, cplx* psi, int i, int j, double theta)
{
    uint64_t N = (uint64_t)1 << n;
    cplx same = cexp(-I * theta), diff = cexp(I * theta);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z)
        psi[z] *= ((((z >> i) ^ (z >> j)) & 1) ? diff : same);
}

/* Eq. (twocomponentupdates) with u = exp(-i beta X) = [[c, -i s], [-i s, c]]:
 * loop over all pairs (z, z + 2^j) with bit j of z clear. */
void orc_gate_x(int n, cplx* psi, int j, double beta)
{
    uint64_t N = (uint64_t)1 << n, bit = (uint64_t)1 << j;
    cplx u00 = cos(beta), u01 = -I * sin(beta), u10 = -I * sin(beta), u11 = cos(beta);
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        if ((uint64_t)z & bit) continue;
        cplx a = psi[z], b = psi[(uint64_t)z | bit];
        psi[z] = u00 * a + u01 * b;
        psi[(uint64_t)z | bit] = u10 * a + u11 * b;
    }
}

/* One QAOA layer: e^{-i beta H_D} e^{-i gamma H_C}, gate by gate. */
void orc_layer(int n, cplx* psi, const double* h, int m, const int32_t* edges, const double* J,
               double gamma, double beta)
{
    for (int i = 0; i < n; ++i) orc_gate_z(n, psi, i, gamma * h[i]);
    for (int e = 0; e < m; ++e) orc_gate_zz(n, psi, edges[2 * e], edges[2 * e + 1], gamma * J[e]);
    for (int i = 0; i < n; ++i) orc_gate_x(n, psi, i, beta);
}

/* Eq. (QAOA_state). from_plus = 1 starts from |+>^n, else continues from psi. */
void orc_evolve(int n, cplx* psi, const double* h, int m, const int32_t* edges, const double* J,
                int p, const double* gamma, const double* beta, int from_plus)
{
    if (from_plus) orc_init_plus(n, psi);
    for (int k = 0; k < p; ++k) orc_layer(n, psi, h, m, edges, J, gamma[k], beta[k]);
}

/* E = sum_z |psi_z|^2 C(z); P = weight on cost == cmin; norm = sum |psi_z|^2. */
void orc_readout(int n, const cplx* psi, const double* h, int m, const int32_t* edges, const double* J,
                 double cmin, double* E_out, double* P_out, double* norm_out)
{
    uint64_t N = (uint64_t)1 << n;
    double E = 0.0, P = 0.0, nrm = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : E, P, nrm)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        double w = creal(psi[z]) * creal(psi[z]) + cimag(psi[z]) * cimag(psi[z]);
        double c = orc_cost(n, h, m, edges, J, (uint64_t)z);
        E += w * c;
        nrm += w;
        if (c == cmin) P += w;
    }
    *E_out = E; *P_out = P; *norm_out = nrm;
}

/* Im <lam| Z_i |psi> */
static double im_z(int n, const cplx* lam, const cplx* psi, int i)
{
    uint64_t N = (uint64_t)1 << n;
    double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (int64_t z = 0; z < (int64_t)N; ++z) acc += spin((uint64_t)z, i) * cimag(conj(lam[z]) * psi[z]);
    return acc;
}

/* Im <lam| Z_i Z_j |psi> */
static double im_zz(int n, const cplx* lam, const cplx* psi, int i, int j)
{
    uint64_t N = (uint64_t)1 << n;
    double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (int64_t z = 0; z < (int64_t)N; ++z)
        acc += spin((uint64_t)z, i) * spin((uint64_t)z, j) * cimag(conj(lam[z]) * psi[z]);
    return acc;
}

/* Im <lam| X_j |psi> */
static double im_x(int n, const cplx* lam, const cplx* psi, int j)
{
    uint64_t N = (uint64_t)1 << n, bit = (uint64_t)1 << j;
    double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (int64_t z = 0; z < (int64_t)N; ++z) acc += cimag(conj(lam[z]) * psi[(uint64_t)z ^ bit]);
    return acc;
}

/*
 * Reverse-mode derivative of F = <psi_p| O |psi_p> with O = H_C
 * (objective 0) or the projector on the minimal-cost states (objective 1).
 * psi and lam are caller-provided work arrays of 2^n entries.
 * Returns F, dF/dgamma_k and dF/dbeta_k for k = 1..p.
 */
void orc_adjoint(int n, const double* h, int m, const int32_t* edges, const double* J,
                 int p, const double* gamma, const double* beta, int objective, double cmin,
                 cplx* psi, cplx* lam, double* value, double* dgamma, double* dbeta)
{
    uint64_t N = (uint64_t)1 << n;
    orc_evolve(n, psi, h, m, edges, J, p, gamma, beta, 1);

    double F = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : F)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        double c = orc_cost(n, h, m, edges, J, (uint64_t)z);
        double o = objective == 0 ? c : (c == cmin ? 1.0 : 0.0);
        lam[z] = o * psi[z];
        F += o * (creal(psi[z]) * creal(psi[z]) + cimag(psi[z]) * cimag(psi[z]));
    }
    *value = F;

    for (int k = p - 1; k >= 0; --k) {
        /* mixer gates of layer k, last applied first undone */
        double gb = 0.0;
        for (int i = n - 1; i >= 0; --i) {
            gb += 2.0 * im_x(n, lam, psi, i);
            orc_gate_x(n, psi, i, -beta[k]);
            orc_gate_x(n, lam, i, -beta[k]);
        }
        dbeta[k] = gb;
        /* coupling phases, then field phases, in reverse */
        double gg = 0.0;
        for (int e = m - 1; e >= 0; --e) {
            int a = edges[2 * e], b = edges[2 * e + 1];
            gg += 2.0 * J[e] * im_zz(n, lam, psi, a, b);
            orc_gate_zz(n, psi, a, b, -gamma[k] * J[e]);
            orc_gate_zz(n, lam, a, b, -gamma[k] * J[e]);
        }
        for (int i = n - 1; i >= 0; --i) {
            gg += 2.0 * h[i] * im_z(n, lam, psi, i);
            orc_gate_z(n, psi, i, -gamma[k] * h[i]);
            orc_gate_z(n, lam, i, -gamma[k] * h[i]);
        }
        dgamma[k] = gg;
    }
}

/*
 * Spin expectation values <Z_i> = sum_z |psi_z|^2 s_i(z), i = 0..n-1, of one
 * state (the per-qubit <sigma^z_i> that the AQA runs record during the time
 * evolution, Sec. III.B.2, shown in Fig. 6).  One plain pass per qubit.
 */
void orc_zexp(int n, const cplx* psi, double* out)
{
    uint64_t N = (uint64_t)1 << n;
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
        for (int64_t z = 0; z < (int64_t)N; ++z) {
            double w = creal(psi[z]) * creal(psi[z]) + cimag(psi[z]) * cimag(psi[z]);
            acc += w * spin((uint64_t)z, i);
        }
        out[i] = acc;
    }
}

/* Eq. (QAOA_state) from |+>^n, recording <Z_i> after every layer:
 * out[k * n + i] for layers k = 0..p-1 (after the mixer of layer k). */
void orc_evolve_zexp(int n, cplx* psi, const double* h, int m, const int32_t* edges, const double* J,
                     int p, const double* gamma, const double* beta, double* out)
{
    orc_init_plus(n, psi);
    for (int k = 0; k < p; ++k) {
        orc_layer(n, psi, h, m, edges, J, gamma[k], beta[k]);
        orc_zexp(n, psi, out + (size_t)k * n);
    }
}

/* Eq. (twocomponentupdates) with a general 2 x 2 matrix u (row major,
 * u = [u00, u01, u10, u11] as re, im pairs): for every pair (z, z + 2^j)
 * with bit j of z clear, (a, b) -> (u00 a + u01 b, u10 a + u11 b). */
void orc_gate_u(int n, cplx* psi, int j, const double* u)
{
    uint64_t N = (uint64_t)1 << n, step = (uint64_t)1 << j;
    const cplx u00 = u[0] + I * u[1], u01 = u[2] + I * u[3], u10 = u[4] + I * u[5], u11 = u[6] + I * u[7];
#pragma omp parallel for schedule(static)
    for (int64_t z = 0; z < (int64_t)N; ++z) {
        if ((uint64_t)z & step) continue;
        cplx a = psi[z], b = psi[(uint64_t)z + step];
        psi[z] = u00 * a + u01 * b;
        psi[(uint64_t)z + step] = u10 * a + u11 * b;
    }
}

/* exp(i theta (a X + b Z)) of one spin: cos(theta r) + i sin(theta r) (a X + b Z) / r,
 * r = sqrt(a^2 + b^2) (the identity when r = 0). */
static void spin_exp(double theta, double a, double b, double* u)
{
    double r = sqrt(a * a + b * b);
    double c = cos(theta * r), sr = r > 0.0 ? sin(theta * r) / r : 0.0;
    cplx u00 = c + I * sr * b, u01 = I * sr * a, u11 = c - I * sr * b;
    u[0] = creal(u00); u[1] = cimag(u00);
    u[2] = creal(u01); u[3] = cimag(u01);
    u[4] = creal(u01); u[5] = cimag(u01);
    u[6] = creal(u11); u[7] = cimag(u11);
}

/*
 * Quantum spin dynamics by the second-order product formula of Eq. (AQA4),
 * step by step as written: for l = 0..nsteps-1,
 *   S_l(tau/2) = exp[i tau/2 sum_i (A_l sigma^x_i - B_l h_i sigma^z_i)],
 *   Z_l(tau)   = exp[-i tau B_l sum_{ij} J_ij sigma^z_i sigma^z_j],
 *   psi <- S_l(tau/2) Z_l(tau) S_l(tau/2) psi,
 * from |+>^n, with the fields of Eq. (AQA3) (h~^x = A, h~^z_i = -B h_i,
 * J~^z_ij = -B J_ij).  Each single-spin exponential is the exact 2 x 2
 * matrix; each coupling an exp(-i theta Z_i Z_j) gate.
 */
void orc_qsds_evolve(int n, cplx* psi, const double* h, int m, const int32_t* edges, const double* J,
                     int nsteps, double tau, const double* A, const double* B)
{
    double u[8];
    orc_init_plus(n, psi);
    for (int l = 0; l < nsteps; ++l) {
        for (int half = 0; half < 2; ++half) {
            for (int i = 0; i < n; ++i) {
                spin_exp(0.5 * tau, A[l], -B[l] * h[i], u);
                orc_gate_u(n, psi, i, u);
            }
            if (half == 0)
                for (int e = 0; e < m; ++e) orc_gate_zz(n, psi, edges[2 * e], edges[2 * e + 1], tau * B[l] * J[e]);
        }
    }
}

/* Host threads used by the OpenMP loops above (timing of the CPU baseline
 * with all cores and with one). */
void orc_set_threads(int t)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

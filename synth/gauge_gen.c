/*
 * Seeded synthetic gauge fields for the Moebius domain-wall solve.
 *
 * Input generation only: random SU(3) links U = exp(i eps H) and the Wilson
 * (gradient) flow used in Sec. III of arXiv:1701.07559 to smooth them
 * (t_gf = 1 in lattice units).  Both the CPU oracle and the GPU library
 * consume these fields; neither side's solver arithmetic lives here.
 *
 * Layout: U[t][z][y][x][mu][a][b], complex interleaved (re, im), mu = x,y,z,t.
 *
 * Random numbers: a counter-based generator (SplitMix64 mixing of
 * (seed, stream, matrix index)), then Box-Muller, so a field does not depend
 * on thread count or order.
 *
 * Flow: dV/dt = Z(V) V with Z = -P_TA(Omega), Omega_mu(x) the sum of the six
 * plaquettes that start with V_mu(x) and P_TA the traceless anti-Hermitian
 * part; integrated with the three-stage Runge-Kutta scheme of Luscher
 * (JHEP 08 (2010) 071), the reference the paper cites for the flow.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

typedef struct { double re, im; } cplx;
typedef struct { cplx m[9]; } mat3;

static inline cplx cadd(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx cmul(cplx a, cplx b) { cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static inline cplx cconj(cplx a) { cplx r = {a.re, -a.im}; return r; }

static void m_mul(const mat3* a, const mat3* b, mat3* c) {
    mat3 t;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = {0.0, 0.0};
            for (int k = 0; k < 3; k++) s = cadd(s, cmul(a->m[3 * i + k], b->m[3 * k + j]));
            t.m[3 * i + j] = s;
        }
    *c = t;
}
/* c = a * b^+ */
static void m_mul_d(const mat3* a, const mat3* b, mat3* c) {
    mat3 t;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = {0.0, 0.0};
            for (int k = 0; k < 3; k++) s = cadd(s, cmul(a->m[3 * i + k], cconj(b->m[3 * j + k])));
            t.m[3 * i + j] = s;
        }
    *c = t;
}
static void m_add(mat3* a, const mat3* b) { for (int i = 0; i < 9; i++) a->m[i] = cadd(a->m[i], b->m[i]); }
static void m_scale(mat3* a, double s) { for (int i = 0; i < 9; i++) { a->m[i].re *= s; a->m[i].im *= s; } }
static void m_id(mat3* a) { memset(a, 0, sizeof(*a)); a->m[0].re = a->m[4].re = a->m[8].re = 1.0; }

/* exp(X) by scaling and squaring of a Taylor series (X small after scaling). */
static void m_exp(const mat3* X, mat3* out) {
    double nrm = 0.0;
    for (int i = 0; i < 9; i++) nrm += X->m[i].re * X->m[i].re + X->m[i].im * X->m[i].im;
    nrm = sqrt(nrm);
    int sq = 0;
    while (nrm > 0.125) { nrm *= 0.5; sq++; }
    mat3 Y = *X;
    m_scale(&Y, ldexp(1.0, -sq));
    mat3 term, sum;
    m_id(&sum);
    m_id(&term);
    for (int k = 1; k <= 18; k++) {
        m_mul(&term, &Y, &term);
        m_scale(&term, 1.0 / k);
        m_add(&sum, &term);
    }
    for (int i = 0; i < sq; i++) m_mul(&sum, &sum, &sum);
    *out = sum;
}

/* ---- counter-based random numbers ---- */
static inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
static inline double u01(uint64_t* state) {
    *state += 0x9E3779B97F4A7C15ull;
    uint64_t z = splitmix64(*state);
    return ((double)(z >> 11) + 1.0) * 0x1.0p-53;   /* in (0, 1] */
}

/* Gell-Mann matrices lambda_a / 2, a = 1..8, accumulated as H = sum w_a lambda_a / 2. */
static void hermitian_from_weights(const double w[8], mat3* H) {
    memset(H, 0, sizeof(*H));
    const double r3 = 1.0 / sqrt(3.0);
    /* lambda1 */ H->m[1].re += 0.5 * w[0]; H->m[3].re += 0.5 * w[0];
    /* lambda2 */ H->m[1].im += -0.5 * w[1]; H->m[3].im += 0.5 * w[1];
    /* lambda3 */ H->m[0].re += 0.5 * w[2]; H->m[4].re += -0.5 * w[2];
    /* lambda4 */ H->m[2].re += 0.5 * w[3]; H->m[6].re += 0.5 * w[3];
    /* lambda5 */ H->m[2].im += -0.5 * w[4]; H->m[6].im += 0.5 * w[4];
    /* lambda6 */ H->m[5].re += 0.5 * w[5]; H->m[7].re += 0.5 * w[5];
    /* lambda7 */ H->m[5].im += -0.5 * w[6]; H->m[7].im += 0.5 * w[6];
    /* lambda8 */ H->m[0].re += 0.5 * r3 * w[7]; H->m[4].re += 0.5 * r3 * w[7];
                  H->m[8].re += -1.0 * r3 * w[7];
}

/* n matrices exp(i eps H_k), H_k = sum_a w_a lambda_a/2, w_a ~ N(0,1) drawn from
 * the counter (seed, stream, k).  out: n * 18 doubles. */
void synth_random_su3(long n, uint64_t seed, uint64_t stream, double eps, double* out) {
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++) {
        uint64_t st = splitmix64(seed ^ splitmix64(stream ^ splitmix64((uint64_t)k)));
        double w[8];
        for (int a = 0; a < 8; a += 2) {
            double u1 = u01(&st), u2 = u01(&st);
            double r = sqrt(-2.0 * log(u1));
            w[a] = r * cos(2.0 * M_PI * u2);
            w[a + 1] = r * sin(2.0 * M_PI * u2);
        }
        mat3 H, X, U;
        hermitian_from_weights(w, &H);
        /* X = i eps H */
        for (int i = 0; i < 9; i++) { X.m[i].re = -eps * H.m[i].im; X.m[i].im = eps * H.m[i].re; }
        m_exp(&X, &U);
        memcpy(out + 18 * k, &U, sizeof(U));
    }
}

/* ---- lattice geometry ---- */
static inline long site_index(const int L[4], int x, int y, int z, int t) {
    return x + (long)L[0] * (y + (long)L[1] * (z + (long)L[2] * t));
}
static inline long neighbour(const int L[4], long s, int mu, int dir) {
    int c[4];
    long r = s;
    for (int i = 0; i < 4; i++) { c[i] = (int)(r % L[i]); r /= L[i]; }
    c[mu] = (c[mu] + dir + L[mu]) % L[mu];
    return site_index(L, c[0], c[1], c[2], c[3]);
}
static inline const mat3* link(const double* U, long s, int mu) { return (const mat3*)(U + 18 * (4 * s + mu)); }

/* Omega_mu(x): the six plaquettes starting with U_mu(x). */
static void omega(const int L[4], const double* U, long s, int mu, mat3* out) {
    mat3 acc, a, b;
    memset(&acc, 0, sizeof(acc));
    const mat3* Umu = link(U, s, mu);
    long xp = neighbour(L, s, mu, +1);
    for (int nu = 0; nu < 4; nu++) {
        if (nu == mu) continue;
        long xn = neighbour(L, s, nu, +1);
        long xm = neighbour(L, s, nu, -1);
        long xpm = neighbour(L, xp, nu, -1);
        /* U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ */
        m_mul(Umu, link(U, xp, nu), &a);
        m_mul_d(&a, link(U, xn, mu), &b);
        m_mul_d(&b, link(U, s, nu), &a);
        m_add(&acc, &a);
        /* U_mu(x) U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu) */
        m_mul_d(Umu, link(U, xpm, nu), &a);
        m_mul_d(&a, link(U, xm, mu), &b);
        m_mul(&b, link(U, xm, nu), &a);
        m_add(&acc, &a);
    }
    *out = acc;
}

/* Z = -P_TA(Omega), P_TA(M) = (M - M^+)/2 - tr(M - M^+)/6. */
static void flow_generator(const mat3* Om, mat3* Z) {
    mat3 t;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx a = Om->m[3 * i + j], b = cconj(Om->m[3 * j + i]);
            t.m[3 * i + j].re = 0.5 * (a.re - b.re);
            t.m[3 * i + j].im = 0.5 * (a.im - b.im);
        }
    double trim = (t.m[0].im + t.m[4].im + t.m[8].im) / 3.0;
    t.m[0].im -= trim; t.m[4].im -= trim; t.m[8].im -= trim;
    for (int i = 0; i < 9; i++) { Z->m[i].re = -t.m[i].re; Z->m[i].im = -t.m[i].im; }
}

static void compute_Z(const int L[4], const double* U, double* Z, double eps) {
    long V = (long)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++)
        for (int mu = 0; mu < 4; mu++) {
            mat3 Om, z;
            omega(L, U, s, mu, &Om);
            flow_generator(&Om, &z);
            m_scale(&z, eps);
            memcpy(Z + 18 * (4 * s + mu), &z, sizeof(z));
        }
}

/* One Runge-Kutta step of size eps (Luscher's third-order scheme):
 *   W1 = exp(Z0/4) W0
 *   W2 = exp(8/9 Z1 - 17/36 Z0) W1
 *   W3 = exp(3/4 Z2 - 8/9 Z1 + 17/36 Z0) W2,   Z_i = eps Z(W_i).  */
static void rk3_step(const int L[4], double* U, double eps, double* Z0, double* Z1, double* Z2) {
    long nlink = 4L * L[0] * L[1] * L[2] * L[3];
    compute_Z(L, U, Z0, eps);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nlink; k++) {
        mat3 X = *(mat3*)(Z0 + 18 * k), E;
        m_scale(&X, 0.25);
        m_exp(&X, &E);
        m_mul(&E, (mat3*)(U + 18 * k), (mat3*)(U + 18 * k));
    }
    compute_Z(L, U, Z1, eps);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nlink; k++) {
        mat3 X, E, a = *(mat3*)(Z1 + 18 * k), b = *(mat3*)(Z0 + 18 * k);
        for (int i = 0; i < 9; i++) {
            X.m[i].re = 8.0 / 9.0 * a.m[i].re - 17.0 / 36.0 * b.m[i].re;
            X.m[i].im = 8.0 / 9.0 * a.m[i].im - 17.0 / 36.0 * b.m[i].im;
        }
        m_exp(&X, &E);
        m_mul(&E, (mat3*)(U + 18 * k), (mat3*)(U + 18 * k));
    }
    compute_Z(L, U, Z2, eps);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nlink; k++) {
        mat3 X, E, a = *(mat3*)(Z2 + 18 * k), b = *(mat3*)(Z1 + 18 * k), c = *(mat3*)(Z0 + 18 * k);
        for (int i = 0; i < 9; i++) {
            X.m[i].re = 0.75 * a.m[i].re - 8.0 / 9.0 * b.m[i].re + 17.0 / 36.0 * c.m[i].re;
            X.m[i].im = 0.75 * a.m[i].im - 8.0 / 9.0 * b.m[i].im + 17.0 / 36.0 * c.m[i].im;
        }
        m_exp(&X, &E);
        m_mul(&E, (mat3*)(U + 18 * k), (mat3*)(U + 18 * k));
    }
}

/* Flow U in place by nsteps steps of size eps.  Returns 0, or -1 on allocation failure. */
int synth_wilson_flow(const int L[4], double* U, double eps, int nsteps) {
    long nlink = 4L * L[0] * L[1] * L[2] * L[3];
    double* Z0 = (double*)malloc(sizeof(double) * 18 * nlink);
    double* Z1 = (double*)malloc(sizeof(double) * 18 * nlink);
    double* Z2 = (double*)malloc(sizeof(double) * 18 * nlink);
    if (!Z0 || !Z1 || !Z2) { free(Z0); free(Z1); free(Z2); return -1; }
    for (int n = 0; n < nsteps; n++) rk3_step(L, U, eps, Z0, Z1, Z2);
    free(Z0); free(Z1); free(Z2);
    return 0;
}

/* Average plaquette  (1/(6V)) sum_{x, mu<nu} Re tr P_{mu nu}(x) / 3. */
double synth_plaquette(const int L[4], const double* U) {
    long V = (long)L[0] * L[1] * L[2] * L[3];
    double total = 0.0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (long s = 0; s < V; s++)
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                mat3 a, b;
                m_mul(link(U, s, mu), link(U, neighbour(L, s, mu, +1), nu), &a);
                m_mul_d(&a, link(U, neighbour(L, s, nu, +1), mu), &b);
                m_mul_d(&b, link(U, s, nu), &a);
                total += a.m[0].re + a.m[4].re + a.m[8].re;
            }
    return total / (3.0 * 6.0 * (double)V);
}

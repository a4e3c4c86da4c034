/*
 * mcg_oracle.c -- plain FP64 CPU oracle for the Feynman-Kac gravity walk.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product path.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Everything is written for a reader checking it against the paper
 * (arXiv:1709.07469): no blocking, no fusion, no reordering beyond the
 * definitions.  Citations name the paper's section / equation.
 */
#include "mcg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., "Parallel random numbers: as easy as  */
/* 1, 2, 3", SC'11): a 10-round Feistel-like bijection of a 128-bit    */
/* counter under a 64-bit key.  The paper (Sec. 2.3) does not name its */
/* generator; Philox keyed by (seed, station, path) is the reading     */
/* taken here.  Round: two 32x32->64 products of counter words 0 and 2 */
/* with the published multipliers, the high halves xor-ed with the     */
/* other two words and the round key; the key advances by the          */
/* published Weyl increments between rounds.                           */
/* ------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += PHILOX_W0;
            k[1] += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void orc_philox_fill(const uint32_t* ctrs, const uint32_t* keys, int64_t n, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i)
        orc_philox4x32_10(ctrs + 4 * i, keys + 2 * i, out + 4 * i);
}

/* Uniform in (0,1) from one 32-bit word.  ubits = 32: (w + 1/2) 2^-32.
 * ubits = 23: ((w >> 9) + 1/2) 2^-23, the grid the single-precision walk
 * uses; both avoid 0 so that log(u) is finite. */
static double uniform_open(uint32_t w, int ubits)
{
    if (ubits == 23) return ((double)(w >> 9) + 0.5) * 0x1p-23;
    return ((double)w + 0.5) * 0x1p-32;
}

/* Box-Muller: two independent N(0,1) from two uniforms (cosine first). */
static void box_muller(double u1, double u2, double* z0, double* z1)
{
    double r = sqrt(-2.0 * log(u1));
    double a = 2.0 * M_PI * u2;
    *z0 = r * cos(a);
    *z1 = r * sin(a);
}

void orc_normals_block(uint64_t seed, uint32_t s, uint32_t p, uint32_t b,
                       uint32_t tag, int ubits, double z[12])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[12];
    for (uint32_t i = 0; i < 3; ++i) {
        uint32_t ctr[4] = {3u * b + i, p, s, tag};
        orc_philox4x32_10(ctr, key, w + 4 * i);
    }
    for (int i = 0; i < 6; ++i)
        box_muller(uniform_open(w[2 * i], ubits), uniform_open(w[2 * i + 1], ubits),
                   &z[2 * i], &z[2 * i + 1]);
}

void orc_normals_fill(uint64_t seed, uint32_t s, uint32_t p, uint32_t b0,
                      int64_t nblocks, uint32_t tag, int ubits, double* z)
{
    for (int64_t i = 0; i < nblocks; ++i)
        orc_normals_block(seed, s, p, b0 + (uint32_t)i, tag, ubits, z + 12 * i);
}

/* ------------------------------------------------------------------ */
/* Closed forms                                                        */
/* ------------------------------------------------------------------ */

/* Homogeneous sphere, Phi with Delta Phi = 4 pi G rho (Phi < 0):
 *   outside: -G M / r;  inside: -G M (3 a^2 - r^2) / (2 a^3). */
double orc_sphere_phi(double G, double rho0, const double c[3], double a, const double x[3])
{
    double dx = x[0] - c[0], dy = x[1] - c[1], dz = x[2] - c[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double M = 4.0 / 3.0 * M_PI * a * a * a * rho0;
    if (r >= a) return -G * M / r;
    return -G * M * (3.0 * a * a - r * r) / (2.0 * a * a * a);
}

/* dPhi/dz of the sphere (z up; positive above the mass). */
double orc_sphere_gz(double G, double rho0, const double c[3], double a, const double x[3])
{
    double dx = x[0] - c[0], dy = x[1] - c[1], dz = x[2] - c[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double M = 4.0 / 3.0 * M_PI * a * a * a * rho0;
    if (r >= a) return G * M * dz / (r * r * r);
    return G * M * dz / (a * a * a);
}

/* log(t + r) with r = |(t, p, q)|, written so that t < 0 loses nothing:
 * t + r = (p^2 + q^2) / (r - t). */
static double log_t_plus_r(double t, double p, double q, double r)
{
    if (t >= 0.0) return log(t + r);
    return log(p * p + q * q) - log(r - t);
}

/* Corner function of the rectangular prism potential (Nagy 1966; the
 * closed form the paper compares against, Sec. 1 and Sec. 4.2):
 *   F = xy ln(z+r) + yz ln(x+r) + zx ln(y+r)
 *       - x^2/2 atan(yz/(xr)) - y^2/2 atan(zx/(yr)) - z^2/2 atan(xy/(zr)).
 * Limits: a term whose polynomial prefactor is 0 is 0 (the "indeterminate
 * form" above source edges, Sec. 4.2). */
static double prism_F(double x, double y, double z)
{
    double r = sqrt(x * x + y * y + z * z);
    if (r == 0.0) return 0.0;
    double f = 0.0;
    if (x * y != 0.0) f += x * y * log_t_plus_r(z, x, y, r);
    if (y * z != 0.0) f += y * z * log_t_plus_r(x, y, z, r);
    if (z * x != 0.0) f += z * x * log_t_plus_r(y, z, x, r);
    if (x != 0.0) f -= 0.5 * x * x * atan(y * z / (x * r));
    if (y != 0.0) f -= 0.5 * y * y * atan(z * x / (y * r));
    if (z != 0.0) f -= 0.5 * z * z * atan(x * y / (z * r));
    return f;
}

/* dF/dz = x ln(y+r) + y ln(x+r) - z atan(xy/(zr)). */
static double prism_dFdz(double x, double y, double z)
{
    double r = sqrt(x * x + y * y + z * z);
    if (r == 0.0) return 0.0;
    double f = 0.0;
    if (x != 0.0) f += x * log_t_plus_r(y, z, x, r);
    if (y != 0.0) f += y * log_t_plus_r(x, y, z, r);
    if (z != 0.0) f -= z * atan(x * y / (z * r));
    return f;
}

/* Triple bracket [[[f]]] = sum over the 8 corners, + at the upper corner,
 * sign flipping with every lower limit, of f(corner - x). */
static double prism_bracket(double (*f)(double, double, double),
                            const double lo[3], const double hi[3], const double x[3])
{
    double s = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k) {
                double cx = (i ? hi[0] : lo[0]) - x[0];
                double cy = (j ? hi[1] : lo[1]) - x[1];
                double cz = (k ? hi[2] : lo[2]) - x[2];
                int nlow = (1 - i) + (1 - j) + (1 - k);
                double sg = (nlow & 1) ? -1.0 : 1.0;
                s += sg * f(cx, cy, cz);
            }
    return s;
}

/* Prism potential Phi = -G rho [[[F]]] (Phi < 0 for rho > 0). */
double orc_prism_phi(double G, double rho0, const double lo[3], const double hi[3], const double x[3])
{
    return -G * rho0 * prism_bracket(prism_F, lo, hi, x);
}

/* dPhi/dx_z of the prism.  The corner offsets are (corner - x), so d/dx_z
 * of F(corner - x) is -dF/dz; with Phi = -G rho [[[F]]] this gives
 * dPhi/dz = +G rho [[[dF/dz]]]. */
double orc_prism_gz(double G, double rho0, const double lo[3], const double hi[3], const double x[3])
{
    return G * rho0 * prism_bracket(prism_dFdz, lo, hi, x);
}

/* ------------------------------------------------------------------ */
/* Density rho(x) and Dirichlet data g(x)                              */
/* ------------------------------------------------------------------ */

/* Piecewise-constant density (Sec. 3: the cube of constant density; the
 * heterogeneous voxel model of the workloads).  Sphere: strict |x-c| < a.
 * Prism and voxel cells: half-open [lo, hi).  Outside the grid: 0. */
double orc_rho(const orc_problem* P, const double x[3])
{
    switch (P->rho_kind) {
    case ORC_RHO_SPHERE: {
        double dx = x[0] - P->center[0], dy = x[1] - P->center[1], dz = x[2] - P->center[2];
        return (dx * dx + dy * dy + dz * dz < P->radius * P->radius) ? P->rho0 : 0.0;
    }
    case ORC_RHO_PRISM:
        for (int k = 0; k < 3; ++k)
            if (!(x[k] >= P->plo[k] && x[k] < P->phi[k])) return 0.0;
        return P->rho0;
    case ORC_RHO_VOXEL: {
        int64_t idx[3];
        for (int k = 0; k < 3; ++k) {
            double t = floor((x[k] - P->origin[k]) / P->spacing[k]);
            if (!(t >= 0.0 && t < (double)P->n[k])) return 0.0;
            idx[k] = (int64_t)t;
        }
        return (double)P->grid[idx[0] + P->n[0] * (idx[1] + P->n[1] * idx[2])];
    }
    default:
        return 0.0;
    }
}

/* Bilinear interpolation in a node-centred table covering the face
 * rectangle [ulo,uhi] x [vlo,vhi] with nu x nv nodes (u fastest). */
static double table_bilinear(const float* t, int32_t nu, int32_t nv,
                             double ulo, double uhi, double vlo, double vhi,
                             double u, double v)
{
    double tu = (u - ulo) / (uhi - ulo) * (double)(nu - 1);
    double tv = (v - vlo) / (vhi - vlo) * (double)(nv - 1);
    double fu = floor(tu), fv = floor(tv);
    if (fu < 0.0) fu = 0.0;
    if (fu > (double)(nu - 2)) fu = (double)(nu - 2);
    if (fv < 0.0) fv = 0.0;
    if (fv > (double)(nv - 2)) fv = (double)(nv - 2);
    int64_t iu = (int64_t)fu, iv = (int64_t)fv;
    double au = tu - fu, av = tv - fv;
    double f00 = t[iu + (int64_t)nu * iv], f10 = t[iu + 1 + (int64_t)nu * iv];
    double f01 = t[iu + (int64_t)nu * (iv + 1)], f11 = t[iu + 1 + (int64_t)nu * (iv + 1)];
    return (1.0 - au) * (1.0 - av) * f00 + au * (1.0 - av) * f10
         + (1.0 - au) * av * f01 + au * av * f11;
}

/* Face index of a boundary point: first axis (lowest index) on which the
 * point lies on lo (face 2k) or hi (face 2k+1); -1 if none. */
static int face_of(const orc_problem* P, const double x[3])
{
    for (int k = 0; k < 3; ++k) {
        if (x[k] == P->lo[k]) return 2 * k;
        if (x[k] == P->hi[k]) return 2 * k + 1;
    }
    return -1;
}

static double g_table(const orc_problem* P, const double x[3], int face)
{
    int k = face / 2;
    int a = (k == 0) ? 1 : 0;          /* u axis: y for x-faces, x otherwise */
    int b = (k == 2) ? 1 : 2;          /* v axis: y for z-faces, z otherwise */
    const float* t = P->faces + (int64_t)face * P->nu * P->nv;
    return table_bilinear(t, P->nu, P->nv, P->lo[a], P->hi[a], P->lo[b], P->hi[b], x[a], x[b]);
}

double orc_g(const orc_problem* P, const double x[3])
{
    switch (P->g_kind) {
    case ORC_G_SPHERE:
        return orc_sphere_phi(P->G, P->rho0, P->center, P->radius, x);
    case ORC_G_PRISM:
        return orc_prism_phi(P->G, P->rho0, P->plo, P->phi, x);
    case ORC_G_TABLE: {
        int f = face_of(P, x);
        if (f < 0) return NAN;
        return g_table(P, x, f);
    }
    case ORC_G_POLY: {
        const double* c = P->poly;
        double X = x[0], Y = x[1], Z = x[2];
        return c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * X + c[5] * Y * Y
             + c[6] * Z * Z + c[7] * X * Y + c[8] * Y * Z + c[9] * Z * X + c[10] * X * Y * Z;
    }
    default:
        return 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* One walk (Sec. 2.3, steps 1-4), with common random numbers          */
/* ------------------------------------------------------------------ */

static int strictly_inside(const orc_problem* P, const double y[3])
{
    if (P->domain_kind == ORC_DOMAIN_BALL) {
        double dx = y[0] - P->bc[0], dy = y[1] - P->bc[1], dz = y[2] - P->bc[2];
        return dx * dx + dy * dy + dz * dz < P->R * P->R;
    }
    for (int k = 0; k < 3; ++k)
        if (!(y[k] > P->lo[k] && y[k] < P->hi[k])) return 0;
    return 1;
}

/* Fraction theta in [0, 1] of the step X -> X + dW at which the segment
 * leaves the ball |x - bc| < R: the positive root of
 * |X - bc + theta dW|^2 = R^2, in the form without cancellation. */
static double ball_theta(const orc_problem* P, const double X[3], const double dW[3])
{
    double a = 0.0, b = 0.0, c = -P->R * P->R;
    for (int k = 0; k < 3; ++k) {
        double q = X[k] - P->bc[k];
        a += dW[k] * dW[k];
        b += 2.0 * q * dW[k];
        c += q * q;
    }
    double D = b * b - 4.0 * a * c;
    double t = (b >= 0.0) ? (-2.0 * c) / (b + sqrt(D)) : (-b + sqrt(D)) / (2.0 * a);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

/* Brownian-bridge exit test of one inside step X -> Y (the paper's Remark on
 * exit-time estimation, after Gobet): for the plane of face k at distances
 * d_X, d_Y the bridge crosses it with probability exp(-2 d_X d_Y / s^2),
 * s = sigma sqrt(dt); the faces are treated as independent, so the step
 * exits with probability 1 - prod_k (1 - p_k).  One uniform per RNG-step,
 * Philox counter (n / 4, p, s, 2) word n % 4, shared by the CRN copies.
 * Returns the face (2k lower, 2k+1 upper) with the largest p_k when the
 * step exits, -1 otherwise. */
static int bridge_exit(const orc_problem* P, const double X[3], const double Y[3], double sd,
                       uint32_t s, uint32_t p, uint32_t n)
{
    double q = 1.0, pmax = -1.0;
    int kmax = -1;
    for (int f = 0; f < 6; ++f) {
        int k = f / 2;
        double dX = (f & 1) ? P->hi[k] - X[k] : X[k] - P->lo[k];
        double dY = (f & 1) ? P->hi[k] - Y[k] : Y[k] - P->lo[k];
        double pk = exp(-2.0 * dX * dY / (sd * sd));
        q *= 1.0 - pk;
        if (pk > pmax) { pmax = pk; kmax = f; }
    }
    uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
    uint32_t ctr[4] = {n / 4u, p, s, 2u}, w[4];
    orc_philox4x32_10(ctr, key, w);
    double U = uniform_open(w[n % 4u], P->ubits);
    return (U < 1.0 - q) ? kmax : -1;
}

int orc_walk_path(const orc_problem* P, const double x0[3], uint32_t s, uint32_t p,
                  double u[3], int64_t steps[3], double xexit[9])
{
    const int nc = P->crn ? 3 : 1;
    const double off[3] = {0.0, P->h, -P->h};
    const double sd = P->sigma * sqrt(P->dt);  /* per-axis step std */
    const double two_pi_G = 2.0 * M_PI * P->G;

    double W[3] = {x0[0], x0[1], x0[2]};      /* the shared Brownian path */
    double I[3] = {0, 0, 0}, rho_prev[3];
    int alive[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) { u[c] = NAN; steps[c] = 0; }
    for (int c = 0; c < nc; ++c) {
        double X[3] = {W[0], W[1], W[2] + off[c]};
        if (!strictly_inside(P, X)) return ORC_ERR_ARG;
        rho_prev[c] = orc_rho(P, X);
        alive[c] = 1;
    }

    double z[12];
    int64_t n = 0;
    for (;;) {
        if (n >= P->max_steps) return ORC_ERR_STEP_CAP;
        if (n % 4 == 0) orc_normals_block(P->seed, s, p, (uint32_t)(n / 4), 0u, P->ubits, z);
        int m = (int)(n % 4);
        /* Step 2: Euler-Maruyama increment (standard Brownian motion,
         * per-axis standard deviation sigma sqrt(dt)). */
        double dW[3] = {sd * z[3 * m], sd * z[3 * m + 1], sd * z[3 * m + 2]};
        double Wn[3] = {W[0] + dW[0], W[1] + dW[1], W[2] + dW[2]};
        int any = 0;
        for (int c = 0; c < nc; ++c) {
            if (!alive[c]) continue;
            double X[3] = {W[0], W[1], W[2] + off[c]};
            double Y[3] = {Wn[0], Wn[1], Wn[2] + off[c]};
            steps[c] += 1;
            if (strictly_inside(P, Y)) {
                int kb = -1;
                if (P->bridge) kb = bridge_exit(P, X, Y, sd, s, p, (uint32_t)n);
                if (kb < 0) {
                    /* Step 3: trapezoid rule for the source integral. */
                    double r = orc_rho(P, Y);
                    I[c] += 0.5 * (rho_prev[c] + r) * P->dt;
                    rho_prev[c] = r;
                    any = 1;
                    continue;
                }
                /* The Brownian bridge between X and Y left Omega through face
                 * kb: the walk ends on that face, below Y, after a full step. */
                double xs[3] = {Y[0], Y[1], Y[2]};
                xs[kb / 2] = (kb & 1) ? P->hi[kb / 2] : P->lo[kb / 2];
                double r = orc_rho(P, xs);
                I[c] += 0.5 * (rho_prev[c] + r) * P->dt;
                u[c] = orc_g(P, xs) - two_pi_G * I[c];
                xexit[3 * c] = xs[0]; xexit[3 * c + 1] = xs[1]; xexit[3 * c + 2] = xs[2];
                alive[c] = 0;
                continue;
            }
            /* Step 4: the walk has left Omega. */
            double xs[3];
            double theta = 1.0;
            if (P->clip && P->domain_kind == ORC_DOMAIN_BALL) {
                /* Clip the last segment where it leaves the ball. */
                theta = ball_theta(P, X, dW);
                for (int k = 0; k < 3; ++k) xs[k] = X[k] + theta * dW[k];
            } else if (P->clip) {
                /* Clip the last segment at the first face it crosses. */
                int kstar = -1;
                double tmin = INFINITY, bstar = 0.0;
                for (int k = 0; k < 3; ++k) {
                    double b;
                    if (Y[k] <= P->lo[k]) b = P->lo[k];
                    else if (Y[k] >= P->hi[k]) b = P->hi[k];
                    else continue;
                    double t = (b - X[k]) / dW[k];
                    if (t < tmin) { tmin = t; kstar = k; bstar = b; }
                }
                if (kstar < 0) return ORC_ERR_ARG;  /* non-finite position */
                theta = tmin;
                if (theta < 0.0) theta = 0.0;
                if (theta > 1.0) theta = 1.0;
                for (int k = 0; k < 3; ++k) xs[k] = X[k] + theta * dW[k];
                xs[kstar] = bstar;
            } else {
                xs[0] = Y[0]; xs[1] = Y[1]; xs[2] = Y[2];
            }
            double r = orc_rho(P, xs);
            I[c] += 0.5 * (rho_prev[c] + r) * theta * P->dt;
            /* Feynman-Kac estimate of this copy (Eq. 5, restated). */
            u[c] = orc_g(P, xs) - two_pi_G * I[c];
            xexit[3 * c] = xs[0]; xexit[3 * c + 1] = xs[1]; xexit[3 * c + 2] = xs[2];
            alive[c] = 0;
        }
        W[0] = Wn[0]; W[1] = Wn[1]; W[2] = Wn[2];
        ++n;
        if (!any) break;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Station statistics (Eq. 7 and the sample variance)                  */
/* ------------------------------------------------------------------ */

/* Neumaier-compensated sum, in index order. */
static double neumaier_sum(const double* v, int64_t n, int64_t stride)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double x = v[i * stride];
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    return s + c;
}

static void mean_and_se(const double* v, int64_t n, double* mean, double* se)
{
    double m = neumaier_sum(v, n, 1) / (double)n;
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = v[i] - m;
        double x = d * d;
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    double m2 = s + c;
    *mean = m;
    *se = (n > 1) ? sqrt(m2 / (double)(n - 1) / (double)n) : NAN;
}

int orc_solve(const orc_problem* P, const double* stations, int64_t S,
              int64_t p0, int64_t N, int nthreads,
              double* u, double* gz, double* se_u, double* se_gz,
              int64_t* path_steps,
              double* pp_u, double* pp_d, int64_t* pp_steps, int64_t* pp_copy_steps)
{
    if (S < 0 || N <= 0 || p0 < 0 || p0 + N > 4294967296LL) return ORC_ERR_ARG;
    if (S == 0) return ORC_OK;
    int64_t total = S * N;
    double* pu = pp_u ? pp_u : (double*)malloc(sizeof(double) * total);
    double* pd = pp_d ? pp_d : (double*)malloc(sizeof(double) * total);
    int64_t* ps = pp_steps ? pp_steps : (int64_t*)malloc(sizeof(int64_t) * total);
    int status = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(max : status)
#endif
    for (int64_t it = 0; it < total; ++it) {
        int64_t s = it / N, i = it % N;
        double uc[3], xe[9];
        int64_t st[3];
        int rc = orc_walk_path(P, stations + 3 * s, (uint32_t)s, (uint32_t)(p0 + i), uc, st, xe);
        if (rc > status) status = rc;
        pu[it] = uc[0];
        pd[it] = P->crn ? (uc[1] - uc[2]) / (2.0 * P->h) : NAN;
        ps[it] = st[0] + st[1] + st[2];
        if (pp_copy_steps) {
            pp_copy_steps[3 * it] = st[0];
            pp_copy_steps[3 * it + 1] = st[1];
            pp_copy_steps[3 * it + 2] = st[2];
        }
    }
    for (int64_t s = 0; s < S; ++s) {
        double m, e;
        mean_and_se(pu + s * N, N, &m, &e);
        if (u) u[s] = m;
        if (se_u) se_u[s] = e;
        mean_and_se(pd + s * N, N, &m, &e);
        if (gz) gz[s] = m;
        if (se_gz) se_gz[s] = e;
        if (path_steps) {
            int64_t t = 0;
            for (int64_t i = 0; i < N; ++i) t += ps[s * N + i];
            path_steps[s] = t;
        }
    }
    if (!pp_u) free(pu);
    if (!pp_d) free(pd);
    if (!pp_steps) free(ps);
    return status;
}

/* ------------------------------------------------------------------ */
/* Heterogeneous model set-up                                          */
/* ------------------------------------------------------------------ */

/* Gaussian random field on an nx*ny*nz voxel grid (x fastest):
 *  1. white noise N(0,1), four voxels per Philox call with counter
 *     (q, 0, 0, 1) for voxels 4q..4q+3, two Box-Muller pairs;
 *  2. separable Gaussian smoothing, std sigma_vox voxels, taps |m| <=
 *     ceil(3 sigma_vox), weights normalised to sum 1, zero outside;
 *  3. rescaled to zero mean and unit (population) standard deviation;
 *  4. rho = amp (exp(Z) - 1). */
void orc_grf_density(uint64_t seed, int64_t nx, int64_t ny, int64_t nz,
                     double sigma_vox, double amp, float* grid_out, double* z_out)
{
    int64_t n = nx * ny * nz;
    double* a = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t q = 0; 4 * q < n; ++q) {
        uint32_t ctr[4] = {(uint32_t)q, 0u, 0u, 1u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double z[4];
        box_muller(uniform_open(w[0], 32), uniform_open(w[1], 32), &z[0], &z[1]);
        box_muller(uniform_open(w[2], 32), uniform_open(w[3], 32), &z[2], &z[3]);
        for (int j = 0; j < 4 && 4 * q + j < n; ++j) a[4 * q + j] = z[j];
    }
    int R = (int)ceil(3.0 * sigma_vox);
    double* wt = (double*)malloc(sizeof(double) * (2 * R + 1));
    double wsum = 0.0;
    for (int m = -R; m <= R; ++m) {
        wt[m + R] = exp(-(double)m * (double)m / (2.0 * sigma_vox * sigma_vox));
        wsum += wt[m + R];
    }
    for (int m = 0; m <= 2 * R; ++m) wt[m] /= wsum;
    int64_t dims[3] = {nx, ny, nz};
    int64_t strides[3] = {1, nx, nx * ny};
    for (int axis = 0; axis < 3; ++axis) {
        int64_t L = dims[axis], st = strides[axis];
        for (int64_t v = 0; v < n; ++v) {
            int64_t coord = (v / st) % L;
            double acc = 0.0;
            for (int m = -R; m <= R; ++m) {
                int64_t c2 = coord + m;
                if (c2 < 0 || c2 >= L) continue;
                acc += wt[m + R] * a[v + m * st];
            }
            b[v] = acc;
        }
        double* t = a; a = b; b = t;
    }
    double mean = neumaier_sum(a, n, 1) / (double)n;
    for (int64_t v = 0; v < n; ++v) b[v] = (a[v] - mean) * (a[v] - mean);
    double sd = sqrt(neumaier_sum(b, n, 1) / (double)n);
    for (int64_t v = 0; v < n; ++v) {
        double Z = (a[v] - mean) / sd;
        if (z_out) z_out[v] = Z;
        grid_out[v] = (float)(amp * (exp(Z) - 1.0));
    }
    free(a); free(b); free(wt);
}

/* Potential at table nodes by direct summation of the prism potential of
 * every voxel (its density taken from the grid), in voxel order. */
int orc_table_nodes(const orc_problem* P, const int64_t* face, const int64_t* iu,
                    const int64_t* iv, int64_t n, int nthreads, double* out)
{
    if (P->rho_kind != ORC_RHO_VOXEL || P->nu < 2 || P->nv < 2) return ORC_ERR_ARG;
    int status = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(max : status)
#endif
    for (int64_t q = 0; q < n; ++q) {
        int f = (int)face[q];
        if (f < 0 || f > 5 || iu[q] < 0 || iu[q] >= P->nu || iv[q] < 0 || iv[q] >= P->nv) {
            status = ORC_ERR_ARG;
            out[q] = NAN;
            continue;
        }
        int k = f / 2;
        int a = (k == 0) ? 1 : 0, b = (k == 2) ? 1 : 2;
        double x[3];
        x[k] = (f & 1) ? P->hi[k] : P->lo[k];
        x[a] = P->lo[a] + (P->hi[a] - P->lo[a]) * (double)iu[q] / (double)(P->nu - 1);
        x[b] = P->lo[b] + (P->hi[b] - P->lo[b]) * (double)iv[q] / (double)(P->nv - 1);
        double s = 0.0, c = 0.0;
        for (int64_t z = 0; z < P->n[2]; ++z)
            for (int64_t y = 0; y < P->n[1]; ++y)
                for (int64_t xx = 0; xx < P->n[0]; ++xx) {
                    double rho = P->grid[xx + P->n[0] * (y + P->n[1] * z)];
                    if (rho == 0.0) continue;
                    double lo[3] = {P->origin[0] + P->spacing[0] * (double)xx,
                                    P->origin[1] + P->spacing[1] * (double)y,
                                    P->origin[2] + P->spacing[2] * (double)z};
                    double hi[3] = {lo[0] + P->spacing[0], lo[1] + P->spacing[1], lo[2] + P->spacing[2]};
                    double v = orc_prism_phi(P->G, rho, lo, hi, x);
                    double t = s + v;
                    if (fabs(s) >= fabs(v)) c += (s - t) + v;
                    else c += (v - t) + s;
                    s = t;
                }
        out[q] = s + c;
    }
    return status;
}

int orc_voxel_field(const orc_problem* P, const double* x, int64_t n, int nthreads, double* phi, double* gz)
{
    if (P->rho_kind != ORC_RHO_VOXEL) return ORC_ERR_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        double s = 0.0, c = 0.0, sg = 0.0, cg = 0.0;
        for (int64_t z = 0; z < P->n[2]; ++z)
            for (int64_t y = 0; y < P->n[1]; ++y)
                for (int64_t xx = 0; xx < P->n[0]; ++xx) {
                    double rho = P->grid[xx + P->n[0] * (y + P->n[1] * z)];
                    if (rho == 0.0) continue;
                    double lo[3] = {P->origin[0] + P->spacing[0] * (double)xx,
                                    P->origin[1] + P->spacing[1] * (double)y,
                                    P->origin[2] + P->spacing[2] * (double)z};
                    double hi[3] = {lo[0] + P->spacing[0], lo[1] + P->spacing[1], lo[2] + P->spacing[2]};
                    double v = orc_prism_phi(P->G, rho, lo, hi, x + 3 * q);
                    double t = s + v;
                    if (fabs(s) >= fabs(v)) c += (s - t) + v;
                    else c += (v - t) + s;
                    s = t;
                    if (gz) {
                        double g = orc_prism_gz(P->G, rho, lo, hi, x + 3 * q);
                        double tg = sg + g;
                        if (fabs(sg) >= fabs(g)) cg += (sg - tg) + g;
                        else cg += (g - tg) + sg;
                        sg = tg;
                    }
                }
        phi[q] = s + c;
        if (gz) gz[q] = sg + cg;
    }
    return ORC_OK;
}

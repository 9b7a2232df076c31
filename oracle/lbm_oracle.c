/*
 * FP64 CPU oracle for the D3Q27 central-Hermite-moment MRT lattice Boltzmann
 * step of "Simulation of the FDA Nozzle Benchmark: A Lattice Boltzmann Study"
 * (arXiv 2204.10566).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never calls it and shares no code, header or table with it.
 *
 * Everything is computed from the definitions, in double precision, without
 * factorisation:
 *   - stencil and weights: 1-D Gauss-Hermite weights 2/3 (c=0) and 1/6 (c=+-1),
 *     3-D weight = product over axes, theta0 = 1/3 (Appendix A, weight eqs.);
 *   - tensor Hermite polynomials by the recursion that generates the paper's
 *     "cyc" forms, H_{a b...}(xi) = xi_a H_{b...} - theta0 sum_k delta_{a k} H_{b..(no k)..}
 *     (Appendix A, Hermite polynomial eqs., dimensional reading: the printed
 *     normalised forms carry theta0 = 1);
 *   - equilibrium as the Hermite sum  w_i sum_n a_n^eq : H_n(c_i) / (n! theta0^n)
 *     with a_n^eq = rho u^{(x)n} (Sec. 2.1 equilibrium eq. read with the order n
 *     in the prefactor; Appendix A equilibrium-coefficient eqs.), restricted to
 *     the 27 tensor components the D3Q27 stencil supports (per-axis degree <= 2);
 *   - the collision f* = f + T^-1 S T (f^eq - f) with T_{m,i} = H_m(c_i - u)
 *     (Sec. 2.1, MRT evolution eq. and central Hermite moment eq.), the inverse
 *     applied by Gaussian elimination with partial pivoting on the dense 27x27 T;
 *   - pull streaming, walls by Bouzidi's interpolated bounce-back (halfway
 *     bounce-back, q = 1/2, unless per-link wall distances are given;
 *     Sec. 2.2 "Simulation details"), and the
 *     non-equilibrium-extrapolation velocity inlet / constant-pressure outlet
 *     (Sec. 2.2 "Simulation details", inlet profile eq.);
 *   - the viscous stress from the pre-collision second-order central Hermite
 *     moments and the strain-rate relation of Appendix A (Sec. 2.2).
 *
 * Compile with -ffp-contract=off (no fused multiply-add contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_Q 27
#define ORC_THETA0 (1.0 / 3.0)

enum { ORC_SOLID = 0, ORC_FLUID = 1, ORC_INLET = 2, ORC_OUTLET = 3 };
enum { ORC_PLUG = 0, ORC_PARABOLIC = 1 };

/* Lattice description for a whole-lattice step.  Dense box storage, box cell
 * b = x + nx*(y + ny*z); populations fin/fout are [b][27]. */
typedef struct {
    const uint8_t *flags;       /* nx*ny*nz: 0 solid, 1 fluid, 2 inlet, 3 outlet */
    int32_t nx, ny, nz, periodic; /* periodic bit mask: 1 = x, 2 = y, 4 = z */
    double omega;               /* rate of the six second-order moments */
    double omega3, omega4, omega5, omega6; /* rates of orders 3..6 (ghosts) */
    double u_in;                /* mean inlet velocity u0 (lattice units) */
    double d_in;                /* inlet diameter d0 (cells) for the parabolic profile */
    double axis_x, axis_y;      /* nozzle axis position (cell-face coordinates) */
    double noise_amp;           /* relative amplitude of the inlet perturbation */
    double rho_out;             /* outlet density */
    uint64_t seed;              /* inlet perturbation seed */
    int32_t profile;            /* ORC_PLUG or ORC_PARABOLIC */
    int32_t nthreads;           /* OpenMP threads (0 = runtime default) */
    int32_t ramp;               /* inlet start-up steps T (0: impulsive start) */
    int32_t reserved;
    const uint8_t *wall_q;      /* optional [b][27]: wall distance q = k/256 of wall link i
                                   of fluid cell b (NULL: q = 1/2 on every link) */
} orc_lattice;

/* ---------------------------------------------------------------- stencil */

/* D3Q27 velocities, i = 9(cz+1) + 3(cy+1) + (cx+1) (Appendix A: third-order
 * quadrature, velocities in {-1,0,1}^3). */
void orc_velocity(int i, int c[3])
{
    c[0] = i % 3 - 1;
    c[1] = (i / 3) % 3 - 1;
    c[2] = i / 9 - 1;
}

/* 3-D weight = product of the 1-D weights 2/3 (c=0), 1/6 (c=+-1) (Appendix A). */
double orc_weight(int i)
{
    int c[3];
    double w = 1.0;
    orc_velocity(i, c);
    for (int a = 0; a < 3; ++a) w *= (c[a] == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
    return w;
}

/* ------------------------------------------------------ Hermite polynomials */

/* Tensor Hermite polynomial H_{idx[0] .. idx[n-1]}(xi) for reference
 * temperature theta0 = 1/3.  Expanding the sum over index pairings (the "cyc"
 * terms of Appendix A) by its first index gives the recursion below. */
double orc_hermite(const int *idx, int n, const double xi[3])
{
    if (n == 0) return 1.0;
    double r = xi[idx[0]] * orc_hermite(idx + 1, n - 1, xi);
    int rest[8];
    for (int k = 1; k < n; ++k) {
        if (idx[k] != idx[0]) continue;
        int m = 0;
        for (int j = 1; j < n; ++j)
            if (j != k) rest[m++] = idx[j];
        r -= ORC_THETA0 * orc_hermite(rest, n - 2, xi);
    }
    return r;
}

/* Moment multi-index m = mx + 3 my + 9 mz  ->  index list x..x y..y z..z. */
static int moment_indices(int m, int idx[6], int deg[3])
{
    deg[0] = m % 3;
    deg[1] = (m / 3) % 3;
    deg[2] = m / 9;
    int n = 0;
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < deg[a]; ++k) idx[n++] = a;
    return n;
}

double orc_hermite_m(int m, const double xi[3])
{
    int idx[6], deg[3];
    int n = moment_indices(m, idx, deg);
    return orc_hermite(idx, n, xi);
}

/* Central Hermite transform T_{m,i} = H_m(c_i - u) (Sec. 2.1, central moment
 * definition), row m over the 27 stencil-supported multi-indices. */
void orc_transform(const double u[3], double *T)
{
    for (int i = 0; i < ORC_Q; ++i) {
        int c[3];
        orc_velocity(i, c);
        double xi[3] = {c[0] - u[0], c[1] - u[1], c[2] - u[2]};
        for (int m = 0; m < ORC_Q; ++m) T[m * ORC_Q + i] = orc_hermite_m(m, xi);
    }
}

/* ------------------------------------------------------------ equilibrium */

static double factorial(int n)
{
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= k;
    return r;
}

/* Hermite polynomials at the lattice nodes, H_m(c_i), and the prefactor
 * multiplicity(m) / (n! theta0^n) of the equilibrium sum; both independent of
 * (rho, u), so they are tabulated once when the library loads. */
static double g_node_hermite[ORC_Q][ORC_Q]; /* [m][i] */
static double g_eq_prefactor[ORC_Q];

__attribute__((constructor)) static void orc_tables_init(void)
{
    for (int m = 0; m < ORC_Q; ++m) {
        int idx[6], deg[3];
        int n = moment_indices(m, idx, deg);
        double mult = factorial(n) / (factorial(deg[0]) * factorial(deg[1]) * factorial(deg[2]));
        g_eq_prefactor[m] = mult / (factorial(n) * pow(ORC_THETA0, n));
        for (int i = 0; i < ORC_Q; ++i) {
            int c[3];
            orc_velocity(i, c);
            double xi[3] = {(double)c[0], (double)c[1], (double)c[2]};
            g_node_hermite[m][i] = orc_hermite(idx, n, xi);
        }
    }
}

/* Discrete equilibrium, Sec. 2.1 equilibrium eq. with a_n^eq = rho u^n
 * (Appendix A): w_i sum_n (1/(n! theta0^n)) a_n^eq : H_n(c_i).  The full
 * contraction over index tuples of order n groups into distinct multi-indices
 * m with multiplicity n!/(mx! my! mz!); only the 27 stencil-supported m are
 * kept (per-axis degree <= 2), which is the full expansion the stencil admits. */
void orc_equilibrium(double rho, const double u[3], double *feq)
{
    double a[ORC_Q];
    for (int m = 0; m < ORC_Q; ++m) {
        int idx[6], deg[3];
        int n = moment_indices(m, idx, deg);
        a[m] = rho;
        for (int k = 0; k < n; ++k) a[m] *= u[idx[k]];
    }
    for (int i = 0; i < ORC_Q; ++i) {
        double s = 0.0;
        for (int m = 0; m < ORC_Q; ++m) s += g_eq_prefactor[m] * a[m] * g_node_hermite[m][i];
        feq[i] = orc_weight(i) * s;
    }
}

/* The same sum written over every ordered index tuple (a_1..a_n), n = 0..6,
 * whose per-axis counts are at most 2: the literal tensor contraction.  Used
 * only to pin orc_equilibrium. */
void orc_equilibrium_tuples(double rho, const double u[3], double *feq)
{
    for (int i = 0; i < ORC_Q; ++i) {
        int c[3];
        orc_velocity(i, c);
        double xi[3] = {(double)c[0], (double)c[1], (double)c[2]};
        double s = 0.0;
        for (int n = 0; n <= 6; ++n) {
            int total = 1;
            for (int k = 0; k < n; ++k) total *= 3;
            double acc = 0.0;
            for (int code = 0; code < total; ++code) {
                int idx[6], cnt[3] = {0, 0, 0}, v = code, ok = 1;
                for (int k = 0; k < n; ++k) {
                    idx[k] = v % 3;
                    v /= 3;
                    if (++cnt[idx[k]] > 2) ok = 0;
                }
                if (!ok) continue;
                double a = rho;
                for (int k = 0; k < n; ++k) a *= u[idx[k]];
                acc += a * orc_hermite(idx, n, xi);
            }
            s += acc / (factorial(n) * pow(ORC_THETA0, n));
        }
        feq[i] = orc_weight(i) * s;
    }
}

/* ---------------------------------------------------------------- algebra */

/* Solve A x = b in place (b <- x) by Gaussian elimination with partial
 * pivoting.  A (n x n, row-major) is overwritten.  Returns 0, or -1 if singular. */
int orc_solve(double *A, double *b, int n)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int r = k + 1; r < n; ++r)
            if (fabs(A[r * n + k]) > best) { best = fabs(A[r * n + k]); p = r; }
        if (best == 0.0) return -1;
        if (p != k) {
            for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            double l = A[r * n + k] / A[k * n + k];
            if (l == 0.0) continue;
            for (int j = k; j < n; ++j) A[r * n + j] -= l * A[k * n + j];
            b[r] -= l * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];
        b[k] = s / A[k * n + k];
    }
    return 0;
}

/* ------------------------------------------------------------- collision */

/* Density and velocity: rho = sum f, rho u = sum c f. */
void orc_moments(const double *f, double mom[4])
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < ORC_Q; ++i) {
        int c[3];
        orc_velocity(i, c);
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += c[a] * f[i];
    }
    mom[0] = rho;
    for (int a = 0; a < 3; ++a) mom[1 + a] = j[a] / rho;
}

/* Relaxation rate of moment m: orders 0 and 1 are conserved (their
 * non-equilibrium part is zero, so the rate is immaterial; omega_cons is
 * exposed only to test that); the six second-order moments relax at omega;
 * orders 3..6 at omega3..omega6 (Appendix A: all ghost rates 1 by default). */
static double rate_of(int m, double omega, const double ghost[4], double omega_cons)
{
    int n = m % 3 + (m / 3) % 3 + m / 9;
    if (n <= 1) return omega_cons;
    if (n == 2) return omega;
    return ghost[n - 3];
}

/* One CHM-MRT collision (Sec. 2.1): f* = f + T^-1 S T (f^eq(rho,u) - f).
 * mom receives the (pre-collision) rho, u.  Returns 0 or -1 (singular T). */
int orc_collide(const double *f, double omega, const double ghost[4], double omega_cons,
                double *fpost, double mom[4])
{
    double T[ORC_Q * ORC_Q], feq[ORC_Q], d[ORC_Q], rhs[ORC_Q];
    orc_moments(f, mom);
    double u[3] = {mom[1], mom[2], mom[3]};
    orc_equilibrium(mom[0], u, feq);
    orc_transform(u, T);
    for (int i = 0; i < ORC_Q; ++i) d[i] = feq[i] - f[i];
    for (int m = 0; m < ORC_Q; ++m) {
        double s = 0.0;
        for (int i = 0; i < ORC_Q; ++i) s += T[m * ORC_Q + i] * d[i];
        rhs[m] = rate_of(m, omega, ghost, omega_cons) * s;
    }
    if (orc_solve(T, rhs, ORC_Q) != 0) return -1;
    for (int i = 0; i < ORC_Q; ++i) fpost[i] = f[i] + rhs[i];
    return 0;
}

/* --------------------------------------------------------- inlet noise */

/* SplitMix64 output function (Steele, Lea and Flood 2014; Vigna's public
 * reference): add the golden-ratio increment, then two xor-shift-multiply rounds. */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Counter-based uniform variate in [-1, 1) for (seed, step, node, component):
 * h = sm(((node << 2) | comp) + sm(step + sm(seed))); U = (h >> 40) 2^-23 - 1.
 * The 24 kept bits make U exact in binary32 and binary64 alike. */
double orc_noise(uint64_t seed, int64_t step, int64_t node, int comp)
{
    uint64_t h = orc_splitmix64(seed);
    h = orc_splitmix64((uint64_t)step + h);
    h = orc_splitmix64((((uint64_t)node << 2) | (uint64_t)comp) + h);
    return (double)(h >> 40) * (1.0 / 8388608.0) - 1.0;
}

/* Prescribed inlet velocity at node (x, y) with inward unit normal n:
 * speed = u0 (plug) or 2 u0 (1 - 4 r^2 / d0^2) (Sec. 2.2 inlet profile eq.),
 * r measured from the nozzle axis at the cell centre, plus the seeded
 * perturbation noise_amp * u0 * U per component, all scaled by the start-up
 * ramp below. */
void orc_inlet_velocity(const orc_lattice *L, int x, int y, int64_t node, int64_t step,
                        const int n[3], double u[3])
{
    double speed = L->u_in;
    if (L->profile == ORC_PARABOLIC) {
        double rx = x + 0.5 - L->axis_x, ry = y + 0.5 - L->axis_y;
        double r2 = rx * rx + ry * ry;
        speed = 2.0 * L->u_in * (1.0 - 4.0 * r2 / (L->d_in * L->d_in));
    }
    for (int a = 0; a < 3; ++a) {
        u[a] = speed * n[a];
        if (L->noise_amp != 0.0) u[a] += L->noise_amp * L->u_in * orc_noise(L->seed, step, node, a);
    }
    /* Start-up (the paper does not state one): with ramp T > 0 the whole
     * prescribed velocity is scaled by the smoothstep r(s) = s^2 (3 - 2 s),
     * s = step / T, while step < T (r rises from 0 to 1 with zero slope at
     * both ends). */
    if (step < L->ramp) {
        double s = (double)step / (double)L->ramp;
        double r = s * s * (3.0 - 2.0 * s);
        for (int a = 0; a < 3; ++a) u[a] *= r;
    }
}

/* ----------------------------------------------------------- lattice step */

static int64_t box_index(const orc_lattice *L, int x, int y, int z)
{
    return (int64_t)x + (int64_t)L->nx * ((int64_t)y + (int64_t)L->ny * z);
}

/* Neighbour coordinate along one axis; returns 0 if it leaves a
 * non-periodic box. */
static int wrap(int v, int n, int periodic)
{
    if (v >= 0 && v < n) return 1;
    return periodic ? 1 : 0;
}

static int flag_at(const orc_lattice *L, int x, int y, int z, int64_t *b)
{
    int ok = wrap(x, L->nx, L->periodic & 1) && wrap(y, L->ny, L->periodic & 2) &&
             wrap(z, L->nz, L->periodic & 4);
    if (!ok) return ORC_SOLID;
    x = (x % L->nx + L->nx) % L->nx;
    y = (y % L->ny + L->ny) % L->ny;
    z = (z % L->nz + L->nz) % L->nz;
    *b = box_index(L, x, y, z);
    return L->flags[*b];
}

/* Interior neighbour of an inlet/outlet node: the unique axis neighbour whose
 * flag is FLUID.  Returns its box index, or -1 if there is none or several. */
int64_t orc_nee_neighbour(const orc_lattice *L, int x, int y, int z, int n[3])
{
    static const int dirs[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    int64_t found = -1;
    int count = 0;
    for (int k = 0; k < 6; ++k) {
        int64_t b = -1;
        int fl = flag_at(L, x + dirs[k][0], y + dirs[k][1], z + dirs[k][2], &b);
        if (fl == ORC_FLUID) {
            ++count;
            found = b;
            for (int a = 0; a < 3; ++a) n[a] = dirs[k][a];
        }
    }
    return count == 1 ? found : -1;
}

/* Pull-stream gather for cell (x,y,z): f_i(x, t+1) = f*_i(x - c_i, t), or,
 * when x - c_i is solid or outside a non-periodic box, the population
 * reflected by the wall that cuts the link between x and x - c_i
 * (Sec. 2.2, Bouzidi's interpolated bounce-back).  With ib the opposite of
 * i (the direction that points from x at the wall) and q in (0, 1] the
 * wall's distance from x as a fraction of the link:
 *   q <  1/2:  f_i(x, t+1) = 2q f*_ib(x, t) + (1 - 2q) f*_ib(x + c_i, t),
 *   q >= 1/2:  f_i(x, t+1) = f*_ib(x, t) / (2q) + (1 - 1/(2q)) f*_i(x, t);
 * q = 1/2 is the halfway bounce-back f*_ib(x, t).  When x + c_i is itself
 * solid the first form has no second point and the halfway value is used. */
static void gather(const orc_lattice *L, const double *fin, int x, int y, int z, double *f)
{
    int64_t self = box_index(L, x, y, z);
    for (int i = 0; i < ORC_Q; ++i) {
        int c[3];
        orc_velocity(i, c);
        int64_t src = -1;
        int fl = flag_at(L, x - c[0], y - c[1], z - c[2], &src);
        if (fl != ORC_SOLID) {
            f[i] = fin[src * ORC_Q + i];
            continue;
        }
        const int ib = ORC_Q - 1 - i;
        double fi = fin[self * ORC_Q + ib];
        if (L->wall_q) {
            const double q = L->wall_q[self * ORC_Q + i] / 256.0;
            if (q < 0.5) {
                int64_t nbr = -1;
                if (flag_at(L, x + c[0], y + c[1], z + c[2], &nbr) != ORC_SOLID)
                    fi = 2.0 * q * fin[self * ORC_Q + ib] + (1.0 - 2.0 * q) * fin[nbr * ORC_Q + ib];
            } else {
                fi = fin[self * ORC_Q + ib] / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * fin[self * ORC_Q + i];
            }
        }
        f[i] = fi;
    }
}

/* One time step t -> t_new = t + 1 over the whole lattice.
 * fin: post-collision populations at t; fout: post-collision populations at
 * t_new; mom (optional, [b][4]): rho, u of every active cell at t_new.
 * Fluid cells: gather + collide.  Inlet/outlet nodes: non-equilibrium
 * extrapolation from the interior neighbour x_f (same step):
 *   f*_i(x_b) = f^eq_i(rho_b, u_b) + f*_i(x_f) - f^eq_i(rho_f, u_f),
 * inlet rho_b = rho_f with u_b prescribed; outlet rho_b = rho_out, u_b = u_f.
 * Returns 0, -1 on an inconsistent flag field, -2 on a singular transform. */
int orc_step(const orc_lattice *L, const double *fin, double *fout, double *mom, int64_t t_new)
{
    const int64_t ncell = (int64_t)L->nx * L->ny * L->nz;
    const double ghost[4] = {L->omega3, L->omega4, L->omega5, L->omega6};
    double *m = mom ? mom : (double *)malloc(sizeof(double) * 4 * (size_t)ncell);
    int err = 0;
    if (!m) return -3;
#ifdef _OPENMP
    const int nt = L->nthreads > 0 ? L->nthreads : omp_get_max_threads();
#endif

#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nt) reduction(| : err)
#endif
    for (int64_t b = 0; b < ncell; ++b) {
        if (L->flags[b] != ORC_FLUID) {
            if (L->flags[b] == ORC_SOLID)
                for (int i = 0; i < ORC_Q; ++i) fout[b * ORC_Q + i] = 0.0;
            continue;
        }
        int x = (int)(b % L->nx), y = (int)((b / L->nx) % L->ny), z = (int)(b / ((int64_t)L->nx * L->ny));
        double f[ORC_Q];
        gather(L, fin, x, y, z, f);
        if (orc_collide(f, L->omega, ghost, 1.0, fout + b * ORC_Q, m + b * 4) != 0) err |= 2;
    }

#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nt) reduction(| : err)
#endif
    for (int64_t b = 0; b < ncell; ++b) {
        int fl = L->flags[b];
        if (fl != ORC_INLET && fl != ORC_OUTLET) continue;
        int x = (int)(b % L->nx), y = (int)((b / L->nx) % L->ny), z = (int)(b / ((int64_t)L->nx * L->ny));
        int n[3];
        int64_t bf = orc_nee_neighbour(L, x, y, z, n);
        if (bf < 0) { err |= 1; continue; }
        double rho_f = m[bf * 4], u_f[3] = {m[bf * 4 + 1], m[bf * 4 + 2], m[bf * 4 + 3]};
        double rho_b, u_b[3];
        if (fl == ORC_INLET) {
            rho_b = rho_f;
            orc_inlet_velocity(L, x, y, b, t_new, n, u_b);
        } else {
            rho_b = L->rho_out;
            for (int a = 0; a < 3; ++a) u_b[a] = u_f[a];
        }
        double feq_b[ORC_Q], feq_f[ORC_Q];
        orc_equilibrium(rho_b, u_b, feq_b);
        orc_equilibrium(rho_f, u_f, feq_f);
        for (int i = 0; i < ORC_Q; ++i)
            fout[b * ORC_Q + i] = feq_b[i] + (fout[bf * ORC_Q + i] - feq_f[i]);
        m[b * 4] = rho_b;
        for (int a = 0; a < 3; ++a) m[b * 4 + 1 + a] = u_b[a];
    }
    if (!mom) free(m);
    if (err & 1) return -1;
    if (err & 2) return -2;
    return 0;
}

/* Viscous stress of one cell from its pre-collision populations f (Sec. 2.2
 * viscous shear stress sigma_ab = rho nu (d_b u_a + d_a u_b), with the
 * strain rate of Appendix A taken from the second-order central Hermite
 * moment, sign as in the non-equilibrium stress):
 *   a_ab = sum_i f_i ((c_ia - u_a)(c_ib - u_b) - theta0 delta_ab),
 *   S_ab = -a_ab / (2 rho theta0 tau),  nu = theta0 (tau - 1/2),  tau = 1/omega,
 *   sigma_ab = 2 rho nu S_ab.
 * Components in the order xx, yy, zz, xy, xz, yz. */
void orc_viscous_stress(const double *f, double omega, double sigma[6])
{
    static const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    double mom[4];
    orc_moments(f, mom);
    const double rho = mom[0], tau = 1.0 / omega, nu = ORC_THETA0 * (tau - 0.5);
    for (int k = 0; k < 6; ++k) {
        double a = 0.0;
        for (int i = 0; i < ORC_Q; ++i) {
            int c[3];
            orc_velocity(i, c);
            double h = (c[pa[k]] - mom[1 + pa[k]]) * (c[pb[k]] - mom[1 + pb[k]]);
            if (pa[k] == pb[k]) h -= ORC_THETA0;
            a += f[i] * h;
        }
        const double S = -a / (2.0 * rho * ORC_THETA0 * tau);
        sigma[k] = 2.0 * rho * nu * S;
    }
}

/* Viscous stress field of the step t -> t+1 that starts from the
 * post-collision state fin at t: every fluid cell's stress from its gathered
 * (pre-collision) populations; an inlet/outlet node takes the stress of its
 * interior partner, whose non-equilibrium part the extrapolation copies.
 * sigma: [b][6], zero at solid cells.  Returns 0, or -1 on a node without
 * a unique interior partner. */
int orc_field_stress(const orc_lattice *L, const double *fin, double *sigma)
{
    const int64_t ncell = (int64_t)L->nx * L->ny * L->nz;
    int err = 0;
    for (int64_t b = 0; b < ncell; ++b) {
        for (int k = 0; k < 6; ++k) sigma[b * 6 + k] = 0.0;
        if (L->flags[b] != ORC_FLUID) continue;
        int x = (int)(b % L->nx), y = (int)((b / L->nx) % L->ny), z = (int)(b / ((int64_t)L->nx * L->ny));
        double f[ORC_Q];
        gather(L, fin, x, y, z, f);
        orc_viscous_stress(f, L->omega, sigma + b * 6);
    }
    for (int64_t b = 0; b < ncell; ++b) {
        int fl = L->flags[b];
        if (fl != ORC_INLET && fl != ORC_OUTLET) continue;
        int x = (int)(b % L->nx), y = (int)((b / L->nx) % L->ny), z = (int)(b / ((int64_t)L->nx * L->ny));
        int n[3];
        int64_t bf = orc_nee_neighbour(L, x, y, z, n);
        if (bf < 0) { err = -1; continue; }
        for (int k = 0; k < 6; ++k) sigma[b * 6 + k] = sigma[bf * 6 + k];
    }
    return err;
}

/* Moments of every active cell of a state (rho, ux, uy, uz per box cell). */
void orc_field_moments(const orc_lattice *L, const double *f, double *mom)
{
    const int64_t ncell = (int64_t)L->nx * L->ny * L->nz;
    for (int64_t b = 0; b < ncell; ++b) {
        if (L->flags[b] == ORC_SOLID) { for (int a = 0; a < 4; ++a) mom[b * 4 + a] = 0.0; continue; }
        orc_moments(f + b * ORC_Q, mom + b * 4);
    }
}

/* Total mass sum rho and momentum sum rho u over active cells, Kahan-compensated. */
void orc_totals(const orc_lattice *L, const double *f, double out[4])
{
    const int64_t ncell = (int64_t)L->nx * L->ny * L->nz;
    double s[4] = {0, 0, 0, 0}, comp[4] = {0, 0, 0, 0};
    for (int64_t b = 0; b < ncell; ++b) {
        if (L->flags[b] == ORC_SOLID) continue;
        double v[4] = {0, 0, 0, 0};
        for (int i = 0; i < ORC_Q; ++i) {
            int c[3];
            orc_velocity(i, c);
            double fi = f[b * ORC_Q + i];
            v[0] += fi;
            for (int a = 0; a < 3; ++a) v[1 + a] += c[a] * fi;
        }
        for (int k = 0; k < 4; ++k) {
            double y = v[k] - comp[k];
            double t = s[k] + y;
            comp[k] = (t - s[k]) - y;
            s[k] = t;
        }
    }
    for (int k = 0; k < 4; ++k) out[k] = s[k];
}

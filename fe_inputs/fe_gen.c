/*
 * Seeded synthetic finite-element inputs for the CG solver and its oracle.
 *
 * This file builds test problems only.  It holds none of the solver's
 * arithmetic (no sparse product, no dot product, no Krylov step): it writes
 * the CSR arrays of two SPD operators and seeded random vectors.  Both the
 * CUDA path and the CPU oracle read what it writes.
 *
 * Operators (unknowns ordered lexicographically, x fastest; idx = i + N*(j + N*k)):
 *   - 7-point Laplacian on an N^3 interior grid with homogeneous Dirichlet
 *     boundaries eliminated: diagonal 6, the six face neighbours -1 (h^2 dropped).
 *   - Trilinear hexahedral (Q1) stiffness matrix of -div(rho grad u) on the unit
 *     cube split into (N+1)^3 cube elements of side h = 1/(N+1); the boundary
 *     nodes carry u = 0 and are eliminated, leaving N^3 unknowns.  The paper
 *     discretises its gravity equation with Q1 elements and Dirichlet
 *     conditions (Sec. 5.1); the element matrix is derived here from the
 *     tensor-product form, see fe_q1().
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: draw(seed, stream, i) = mix(mix(seed ^ stream*G) + (i+1)*G) with
 * G = 0x9E3779B97F4A7C15 and mix the SplitMix64 output function.  Uniform
 * doubles take the top 53 bits; normal deviates use the Box-Muller transform
 * (Box & Muller 1958) on two uniforms of consecutive counters.
 */
#include <stdint.h>
#include <math.h>
#include <string.h>

#define FE_GOLDEN 0x9E3779B97F4A7C15ULL

static uint64_t fe_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t fe_draw_u64(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t key = fe_mix64(seed ^ (stream * FE_GOLDEN));
    return fe_mix64(key + (i + 1) * FE_GOLDEN);
}

/* Uniform in [0, 1) with 53 random bits. */
static double fe_u01(uint64_t seed, uint64_t stream, uint64_t i) {
    return (double)(fe_draw_u64(seed, stream, i) >> 11) * 0x1.0p-53;
}

/* out[i] = lo + (hi - lo) * U_i,  U_i uniform in [0,1) from counter i. */
void fe_uniform(uint64_t seed, uint64_t stream, int64_t n, double lo, double hi, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * fe_u01(seed, stream, (uint64_t)i);
}

/* out[i] = N(0,1) deviate i: Box-Muller on the uniforms of counters 2i, 2i+1. */
void fe_normal(uint64_t seed, uint64_t stream, int64_t n, double* out) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < n; ++i) {
        double u1 = 1.0 - fe_u01(seed, stream, 2 * (uint64_t)i);   /* in (0, 1] */
        double u2 = fe_u01(seed, stream, 2 * (uint64_t)i + 1);
        out[i] = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    }
}

/* ---------------------------------------------------------------- 7-point */

int64_t fe_laplace7_nnz(int64_t N) {
    if (N <= 0) return 0;
    return 7 * N * N * N - 6 * N * N;
}

/* Writes row_ptr[N^3+1], col_idx[nnz], val[nnz] (0-based, columns ascending).
 * Returns nnz, or -1 if the sizes do not fit int32 indices. */
int64_t fe_laplace7(int64_t N, int32_t* row_ptr, int32_t* col_idx, double* val) {
    int64_t n = N * N * N, nnz = fe_laplace7_nnz(N);
    if (N < 0 || nnz > INT32_MAX || n > INT32_MAX) return -1;
    int64_t k_out = 0;
    row_ptr[0] = 0;
    for (int64_t k = 0; k < N; ++k)
        for (int64_t j = 0; j < N; ++j)
            for (int64_t i = 0; i < N; ++i) {
                int64_t row = i + N * (j + N * k);
                /* neighbours in ascending column order: -z, -y, -x, self, +x, +y, +z */
                if (k > 0)     { col_idx[k_out] = (int32_t)(row - N * N); val[k_out++] = -1.0; }
                if (j > 0)     { col_idx[k_out] = (int32_t)(row - N);     val[k_out++] = -1.0; }
                if (i > 0)     { col_idx[k_out] = (int32_t)(row - 1);     val[k_out++] = -1.0; }
                col_idx[k_out] = (int32_t)row; val[k_out++] = 6.0;
                if (i < N - 1) { col_idx[k_out] = (int32_t)(row + 1);     val[k_out++] = -1.0; }
                if (j < N - 1) { col_idx[k_out] = (int32_t)(row + N);     val[k_out++] = -1.0; }
                if (k < N - 1) { col_idx[k_out] = (int32_t)(row + N * N); val[k_out++] = -1.0; }
                row_ptr[row + 1] = (int32_t)k_out;
            }
    return k_out;
}

/* ---------------------------------------------------------------- Q1 hex */

int64_t fe_q1_nnz(int64_t N) {
    if (N <= 0) return 0;
    int64_t m = 3 * N - 2;
    return m * m * m;
}

/* Per-element densities rho_e = exp(sigma * Z_e), Z_e ~ N(0,1) drawn from
 * (seed, stream) at the lexicographic element index e = ex + E*(ey + E*ez),
 * E = N+1.  sigma = 0 gives rho = 1 exactly. */
void fe_q1_rho(int64_t N, double sigma, uint64_t seed, uint64_t stream, double* rho) {
    int64_t E = N + 1, ne = E * E * E;
    fe_normal(seed, stream, ne, rho);
    for (int64_t e = 0; e < ne; ++e) rho[e] = exp(sigma * rho[e]);
}

/*
 * Q1 stiffness with element densities rho[(N+1)^3] (from fe_q1_rho or given).
 *
 * For a cube element of side h the trilinear element matrix is
 *   K_e = rho_e * (K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1)
 * with the 1-D element matrices K1 = (1/h)[[1,-1],[-1,1]] and
 * M1 = (h/6)[[2,1],[1,2]].  Two local nodes that differ in d coordinates get
 *   d = 0: h/3,   d = 1: 0,   d = 2: -h/12,   d = 3: -h/12
 * (d = 1: -1/9 + 1/18 + 1/18 = 0 exactly; d = 2: -1/18 - 1/18 + 1/36;
 *  d = 3: 3 * (-1/36)).  A global entry between nodes I and J sums this over
 * the elements holding both nodes: 8 for I = J, 2 for an edge neighbour,
 * 1 for a corner neighbour.  Face-neighbour entries are therefore exactly
 * zero for cube elements whatever rho is; they are stored as explicit 0.0 so
 * that every interior row keeps the full 27-entry pattern (max row length 27,
 * as in the paper's Table 1).  Sums over elements run in lexicographic element
 * order, which makes the matrix bitwise symmetric.
 * Returns nnz, or -1 if the sizes do not fit int32 indices.
 */
int64_t fe_q1(int64_t N, const double* rho, int32_t* row_ptr, int32_t* col_idx, double* val) {
    int64_t n = N * N * N, nnz = fe_q1_nnz(N);
    if (N < 0 || nnz > INT32_MAX || n > INT32_MAX) return -1;
    const int64_t E = N + 1;
    const double h = 1.0 / (double)(N + 1);
    const double c_diag = h / 3.0, c_off = -h / 12.0;
    int64_t k_out = 0;
    row_ptr[0] = 0;
    for (int64_t k = 0; k < N; ++k)
        for (int64_t j = 0; j < N; ++j)
            for (int64_t i = 0; i < N; ++i) {
                int64_t row = i + N * (j + N * k);
                /* node (i,j,k) of the unknown grid is node (i+1,j+1,k+1) of the
                 * full grid; the elements touching it have indices
                 * (i or i+1, j or j+1, k or k+1) in the element grid. */
                for (int dz = -1; dz <= 1; ++dz) {
                    int64_t kk = k + dz;
                    if (kk < 0 || kk >= N) continue;
                    for (int dy = -1; dy <= 1; ++dy) {
                        int64_t jj = j + dy;
                        if (jj < 0 || jj >= N) continue;
                        for (int dx = -1; dx <= 1; ++dx) {
                            int64_t ii = i + dx;
                            if (ii < 0 || ii >= N) continue;
                            int d = (dx != 0) + (dy != 0) + (dz != 0);
                            double v;
                            if (d == 1) {
                                v = 0.0;
                            } else {
                                /* Elements holding both nodes, per axis: offset 0 ->
                                 * {i, i+1}; offset -1 -> {i}; offset +1 -> {i+1}. */
                                int64_t ex0 = (dx == 0) ? i : (dx < 0 ? i : i + 1);
                                int64_t ex1 = (dx == 0) ? i + 1 : ex0;
                                int64_t ey0 = (dy == 0) ? j : (dy < 0 ? j : j + 1);
                                int64_t ey1 = (dy == 0) ? j + 1 : ey0;
                                int64_t ez0 = (dz == 0) ? k : (dz < 0 ? k : k + 1);
                                int64_t ez1 = (dz == 0) ? k + 1 : ez0;
                                double s = 0.0;
                                for (int64_t ez = ez0; ez <= ez1; ++ez)
                                    for (int64_t ey = ey0; ey <= ey1; ++ey)
                                        for (int64_t ex = ex0; ex <= ex1; ++ex)
                                            s += rho[ex + E * (ey + E * ez)];
                                v = (d == 0 ? c_diag : c_off) * s;
                            }
                            col_idx[k_out] = (int32_t)(ii + N * (jj + N * kk));
                            val[k_out++] = v;
                        }
                    }
                }
                row_ptr[row + 1] = (int32_t)k_out;
            }
    return k_out;
}

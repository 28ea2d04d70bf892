/*
 * raftgp_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU restatement of RaftGP's hot path
 * (Gao et al., "RaftGP: Random Fast Graph Partitioning", HPEC 2023):
 *   random feature extraction   (Section III-A, Eq. 5)
 *   random GCN embedding        (Section III-B, Eq. 6 and the row l2-normalisation)
 *   model selection over K      (Section III-C; k-means, scored by Eq. 1 / Eq. 3 / Eq. 7)
 * It exists to check the CUDA library.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never does.  It shares no code,
 * header or table with the CUDA sources.  Every loop follows the definition it cites, in
 * the order the definition states, without blocking, fusion or reordering.
 *
 * Threads: where the iterations of a loop over rows or points are independent (each writes
 * only its own row, point or cluster), the loop may be shared among OpenMP threads; every
 * sum keeps its sequential order (per-point values are summed afterwards in index order,
 * integer counts are exact), so every result is bit-identical for any thread count.
 * orc_set_threads(1) runs everything on one thread.
 *
 * Conventions shared with the library by DEFINITION (each side writes its own code):
 *   - CSR: row_ptr int64[n+1], col int32[nnz]; symmetric, no self loops, no duplicates.
 *   - Degrees d_i = row_ptr[i+1]-row_ptr[i]; 2e = sum_i d_i = nnz.
 *   - d^-1/2 := 0 for an isolated node.
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = 64-bit seed
 *     (low word first), counter words as documented per stream below.
 *   - Gaussians by Box-Muller on 24-bit uniforms u = ((x >> 8) + 0.5) * 2^-24.
 *
 * Readings of the paper taken here (where it is silent or ambiguous):
 *   - Theta_ir ~ N(0, 1/L): variance 1/L, the Johnson-Lindenstrauss scale (Eq. 5 prints
 *     N(0, L^-0.5)).
 *   - Y itself is not row-normalised; every GCN output Z^(k), k >= 1, is (Section III-B).
 *   - tanh in every layer, no bias (Eq. 6); a zero row stays zero under normalisation.
 *   - GCN weights Xavier-normal, std sqrt(2/(L_{k-1}+L_k)) (the paper only says "random").
 *   - k-means: k-means++ seeding by D^2 sampling on 2^-40 fixed-point D^2, Lloyd iterations
 *     with ties to the lowest centroid, an empty cluster keeps its centroid, stop when no
 *     label changes or after T assignment passes.
 *   - Modularity evaluated as Eq. 7 with U = V: sum_r [m_r/e - (vol_r/2e)^2], computed
 *     exactly as the integer ratio (2*(2e)*sum m_r - sum vol_r^2) / (2e)^2 with one
 *     final FP64 division.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

enum { ORC_OP_NCUT = 0, ORC_OP_MOD_FULL = 1, ORC_OP_MOD_REDUCED = 2 };
enum { ORC_CRIT_MOD = 0, ORC_CRIT_NCUT = 1 };

/* Number of threads for the parallel loops (n <= 0: one per processor); returns the count in
 * effect, 1 when the oracle was built without OpenMP. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* 1 when the parallel loops were compiled with OpenMP. */
int orc_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* Counter word 3 of each random stream. */
#define ORC_STREAM_THETA 0x54686574u   /* "Thet" */
#define ORC_STREAM_W 0x57676e6eu       /* "Wgnn" */
#define ORC_STREAM_KMPP 0x4b6d7070u    /* "Kmpp" */

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 S-box with a Weyl key    */
/* schedule.                                                                             */
/* ------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_stream(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

static double uniform24(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

/* Box-Muller: two independent N(0,1) from two uniforms. */
static void box_muller(uint32_t a, uint32_t b, double* g0, double* g1) {
    const double two_pi = 6.283185307179586476925286766559;
    double r = sqrt(-2.0 * log(uniform24(a)));
    double t = two_pi * uniform24(b);
    *g0 = r * cos(t);
    *g1 = r * sin(t);
}

/* Four N(0,1) values from one Philox block. */
static void gauss4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double g[4]) {
    uint32_t x[4];
    philox_stream(seed, c0, c1, c2, c3, x);
    box_muller(x[0], x[1], &g[0], &g[1]);
    box_muller(x[2], x[3], &g[2], &g[3]);
}

/* Eq. 5: Theta in R^{N x L}, Theta_jr ~ N(0, 1/L).  Row j, columns 4q..4q+3 come from
 * the Philox block with counter (q, j_lo, j_hi, "Thet").  `rows` (may be NULL = all
 * rows 0..n_rows-1) lists which rows to produce, so that a sample of a large graph can
 * be generated without the whole matrix. */
void orc_theta_rows(const int64_t* rows, int64_t n_rows, int L, uint64_t seed, double* theta) {
    double sigma = 1.0 / sqrt((double)L);
    for (int64_t t = 0; t < n_rows; ++t) {
        int64_t j = rows ? rows[t] : t;
        for (int q = 0; 4 * q < L; ++q) {
            double g[4];
            gauss4(seed, (uint32_t)q, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), ORC_STREAM_THETA, g);
            for (int s = 0; s < 4 && 4 * q + s < L; ++s) theta[t * L + 4 * q + s] = sigma * g[s];
        }
    }
}

/* GCN weight W^(k) in R^{L_{k-1} x L_k} (row-major), Xavier-normal:
 * W_ab = sqrt(2/(L_{k-1}+L_k)) * g, g from the Philox block (b/4, a, k, "Wgnn"). */
void orc_gcn_weight(int layer, int lin, int lout, uint64_t seed, double* W) {
    double s = sqrt(2.0 / (double)(lin + lout));
    for (int a = 0; a < lin; ++a)
        for (int q = 0; 4 * q < lout; ++q) {
            double g[4];
            gauss4(seed, (uint32_t)q, (uint32_t)a, (uint32_t)layer, ORC_STREAM_W, g);
            for (int t = 0; t < 4 && 4 * q + t < lout; ++t) W[(int64_t)a * lout + 4 * q + t] = s * g[t];
        }
}

/* ------------------------------------------------------------------------------------ */
/* Graph checks and degrees                                                              */
/* ------------------------------------------------------------------------------------ */
int orc_check_csr(int64_t n, const int64_t* row_ptr, const int32_t* col) {
    if (n < 0 || row_ptr[0] != 0) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return ORC_EINVAL;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            if (col[p] < 0 || col[p] >= n || col[p] == i) return ORC_EINVAL;
    }
    return ORC_OK;
}

static int64_t degree(const int64_t* row_ptr, int64_t i) { return row_ptr[i + 1] - row_ptr[i]; }

/* ------------------------------------------------------------------------------------ */
/* Section III-A, Eq. 5: Y = X Theta for X in {M, Q (full), Q-tilde}                      */
/* ------------------------------------------------------------------------------------ */
/* M = D^-1/2 A D^-1/2 (the NCut operator, Eq. 2).
 * Q = A - d d^T / 2e (the modularity matrix, Eq. 4), applied as A Theta - d (d^T Theta) / 2e:
 *     the same matrix product written as a sparse product plus a rank-one term, never
 *     forming the dense N x N matrix.
 * Q-tilde: Q restricted to the edges of G (Section III-A), Q-tilde_ij = 1 - d_i d_j / 2e on
 *     (i,j) in E, 0 elsewhere. */
int orc_project(int64_t n, const int64_t* row_ptr, const int32_t* col, int op, const double* theta,
                int L, double* Y) {
    double two_e = (double)row_ptr[n];
    for (int64_t i = 0; i < n * L; ++i) Y[i] = 0.0;
    if (op == ORC_OP_NCUT) {
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) {
            int64_t di = degree(row_ptr, i);
            if (di == 0) continue;
            double ri = 1.0 / sqrt((double)di);
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                int64_t j = col[p];
                double mij = ri * (1.0 / sqrt((double)degree(row_ptr, j)));
                for (int r = 0; r < L; ++r) Y[i * L + r] += mij * theta[j * L + r];
            }
        }
        return ORC_OK;
    }
    if (op == ORC_OP_MOD_FULL) {
        double* g = (double*)calloc((size_t)L, sizeof(double));
        if (!g) return ORC_ENOMEM;
        for (int64_t j = 0; j < n; ++j)          /* g = d^T Theta */
            for (int r = 0; r < L; ++r) g[r] += (double)degree(row_ptr, j) * theta[j * L + r];
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                for (int r = 0; r < L; ++r) Y[i * L + r] += theta[(int64_t)col[p] * L + r];
            if (two_e > 0.0) {
                double di = (double)degree(row_ptr, i);
                for (int r = 0; r < L; ++r) Y[i * L + r] -= di * g[r] / two_e;
            }
        }
        free(g);
        return ORC_OK;
    }
    if (op == ORC_OP_MOD_REDUCED) {
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) {
            double di = (double)degree(row_ptr, i);
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                int64_t j = col[p];
                double qij = 1.0 - di * (double)degree(row_ptr, j) / two_e;
                for (int r = 0; r < L; ++r) Y[i * L + r] += qij * theta[j * L + r];
            }
        }
        return ORC_OK;
    }
    return ORC_EINVAL;
}

/* ------------------------------------------------------------------------------------ */
/* Section III-B, Eq. 6: Z_out = rownorm(tanh(D^-1/2 (A+I) D^-1/2 Z_in W))                 */
/* with D-hat the degree matrix of A + I, i.e. d-hat_i = d_i + 1.                          */
/* ------------------------------------------------------------------------------------ */
int orc_gcn_layer(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* Zin, int lin,
                  const double* W, int lout, double* Zout) {
    int rc = ORC_OK;
#pragma omp parallel
    {
    double* agg = (double*)malloc(sizeof(double) * (size_t)lin);
    double* h = (double*)malloc(sizeof(double) * (size_t)lout);
    if (!agg || !h) {
#pragma omp atomic write
        rc = ORC_ENOMEM;
    }
#pragma omp for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        if (!agg || !h) continue;
        double rhi = 1.0 / sqrt((double)(degree(row_ptr, i) + 1));
        /* (A-hat_n Z_in)_i = sum over {i} U N(i) of rhi * rhj * Z_in[j] */
        for (int a = 0; a < lin; ++a) agg[a] = rhi * rhi * Zin[i * lin + a];
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int64_t j = col[p];
            double rhj = 1.0 / sqrt((double)(degree(row_ptr, j) + 1));
            for (int a = 0; a < lin; ++a) agg[a] += rhi * rhj * Zin[j * lin + a];
        }
        /* times W^(k), then the activation */
        double norm2 = 0.0;
        for (int b = 0; b < lout; ++b) {
            double s = 0.0;
            for (int a = 0; a < lin; ++a) s += agg[a] * W[(int64_t)a * lout + b];
            h[b] = tanh(s);
            norm2 += h[b] * h[b];
        }
        /* row-wise l2 normalisation; a zero row stays zero */
        double inv = norm2 > 0.0 ? 1.0 / sqrt(norm2) : 0.0;
        for (int b = 0; b < lout; ++b) Zout[i * lout + b] = h[b] * inv;
    }
    free(agg);
    free(h);
    }
    return rc;
}

/* Rows `rows` of Y = X Theta (Eq. 5) for a large graph, drawing the Theta rows of each
 * listed row's neighbours on demand instead of forming Theta.  For the full modularity matrix
 * g = d^T Theta is accumulated over every node, one Theta row at a time. */
int orc_project_rows(int64_t n, const int64_t* row_ptr, const int32_t* col, int op, int L, uint64_t seed,
                     const int64_t* rows, int64_t n_rows, double* Y) {
    double two_e = (double)row_ptr[n];
    const int64_t blk = 4096;
    double* thb = (double*)malloc(sizeof(double) * (size_t)(blk * L));
    double* g = (double*)calloc((size_t)L, sizeof(double));
    if (!thb || !g) { free(thb); free(g); return ORC_ENOMEM; }
    if (op == ORC_OP_MOD_FULL) {
        /* g = d^T Theta over j ascending; the Theta rows of a block are drawn in parallel first */
        for (int64_t j0 = 0; j0 < n; j0 += blk) {
            const int64_t nb = n - j0 < blk ? n - j0 : blk;
#pragma omp parallel for schedule(static)
            for (int64_t t = 0; t < nb; ++t) {
                int64_t j = j0 + t;
                orc_theta_rows(&j, 1, L, seed, thb + t * L);
            }
            for (int64_t t = 0; t < nb; ++t)
                for (int r = 0; r < L; ++r) g[r] += (double)degree(row_ptr, j0 + t) * thb[t * L + r];
        }
    }
    free(thb);
    int rc = ORC_OK;
#pragma omp parallel
    {
    double* th = (double*)malloc(sizeof(double) * (size_t)L);
    if (!th) {
#pragma omp atomic write
        rc = ORC_ENOMEM;
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < n_rows; ++t) {
        if (!th) continue;
        int64_t i = rows[t];
        double di = (double)degree(row_ptr, i);
        double* y = Y + t * L;
        for (int r = 0; r < L; ++r) y[r] = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int64_t j = col[p];
            double dj = (double)degree(row_ptr, j);
            double w;
            if (op == ORC_OP_NCUT) w = (1.0 / sqrt(di)) * (1.0 / sqrt(dj));
            else if (op == ORC_OP_MOD_FULL) w = 1.0;
            else w = 1.0 - di * dj / two_e;
            orc_theta_rows(&j, 1, L, seed, th);
            for (int r = 0; r < L; ++r) y[r] += w * th[r];
        }
        if (op == ORC_OP_MOD_FULL && two_e > 0.0)
            for (int r = 0; r < L; ++r) y[r] -= di * g[r] / two_e;
    }
    free(th);
    }
    free(g);
    if (rc != ORC_OK) return rc;
    return (op >= ORC_OP_NCUT && op <= ORC_OP_MOD_REDUCED) ? ORC_OK : ORC_EINVAL;
}

/* Rows `rows` of one GCN layer (Eq. 6 and the row normalisation) from a given single-precision
 * input Zin (n x lin), each value widened to FP64. */
int orc_gcn_rows(int64_t n, const int64_t* row_ptr, const int32_t* col, const float* Zin, int lin, const double* W,
                 int lout, const int64_t* rows, int64_t n_rows, double* Zout) {
    (void)n;
    int rc = ORC_OK;
#pragma omp parallel
    {
    double* agg = (double*)malloc(sizeof(double) * (size_t)lin);
    double* h = (double*)malloc(sizeof(double) * (size_t)lout);
    if (!agg || !h) {
#pragma omp atomic write
        rc = ORC_ENOMEM;
    }
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < n_rows; ++t) {
        if (!agg || !h) continue;
        int64_t i = rows[t];
        double rhi = 1.0 / sqrt((double)(degree(row_ptr, i) + 1));
        for (int a = 0; a < lin; ++a) agg[a] = rhi * rhi * (double)Zin[i * lin + a];
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int64_t j = col[p];
            double rhj = 1.0 / sqrt((double)(degree(row_ptr, j) + 1));
            for (int a = 0; a < lin; ++a) agg[a] += rhi * rhj * (double)Zin[j * lin + a];
        }
        double norm2 = 0.0;
        for (int b = 0; b < lout; ++b) {
            double sacc = 0.0;
            for (int a = 0; a < lin; ++a) sacc += agg[a] * W[(int64_t)a * lout + b];
            h[b] = tanh(sacc);
            norm2 += h[b] * h[b];
        }
        double inv = norm2 > 0.0 ? 1.0 / sqrt(norm2) : 0.0;
        for (int b = 0; b < lout; ++b) Zout[t * lout + b] = h[b] * inv;
    }
    free(agg);
    free(h);
    }
    return rc;
}

/* Whole embedding: Y = X Theta, then n_layers GCN layers with widths dims[1..n_layers]
 * (dims[0] = L); with n_layers = 0, Z = rownorm(Y).  theta_in / W_in may be NULL (then drawn from `seed`); W_in, when given,
 * is the concatenation of the row-major W^(1..n_layers).  Y_out may be NULL. */
int orc_embed(int64_t n, const int64_t* row_ptr, const int32_t* col, int op, int n_layers, const int* dims,
              uint64_t seed, const double* theta_in, const double* W_in, double* Y_out, double* Z_out) {
    int L = dims[0];
    int maxw = L;
    for (int k = 1; k <= n_layers; ++k) if (dims[k] > maxw) maxw = dims[k];
    double* theta = NULL;
    double* a = (double*)malloc(sizeof(double) * (size_t)(n * maxw + 1));
    double* b = (double*)malloc(sizeof(double) * (size_t)(n * maxw + 1));
    if (!a || !b) { free(a); free(b); return ORC_ENOMEM; }
    if (!theta_in) {
        theta = (double*)malloc(sizeof(double) * (size_t)(n * L + 1));
        if (!theta) { free(a); free(b); return ORC_ENOMEM; }
        orc_theta_rows(NULL, n, L, seed, theta);
        theta_in = theta;
    }
    int rc = orc_project(n, row_ptr, col, op, theta_in, L, a);
    free(theta);
    if (rc) { free(a); free(b); return rc; }
    if (Y_out) memcpy(Y_out, a, sizeof(double) * (size_t)(n * L));
    const double* wp = W_in;
    for (int k = 1; k <= n_layers && rc == ORC_OK; ++k) {
        int lin = dims[k - 1], lout = dims[k];
        double* W = NULL;
        const double* Wk = wp;
        if (!W_in) {
            W = (double*)malloc(sizeof(double) * (size_t)lin * (size_t)lout);
            if (!W) { rc = ORC_ENOMEM; break; }
            orc_gcn_weight(k, lin, lout, seed, W);
            Wk = W;
        } else {
            wp += (size_t)lin * (size_t)lout;
        }
        rc = orc_gcn_layer(n, row_ptr, col, a, lin, Wk, lout, b);
        free(W);
        double* t = a; a = b; b = t;
    }
    if (rc == ORC_OK && n_layers == 0) {
        /* the "w/o Emb" ablation (Table IV): no GCN layer, so the model selection receives the
         * random features themselves, row-normalised as every GCN output is (a zero row stays
         * zero): the ablation removes the layers, not the normalised input of Section III-C */
        for (int64_t i = 0; i < n; ++i) {
            double s2 = 0.0;
            for (int r = 0; r < L; ++r) s2 += a[i * L + r] * a[i * L + r];
            double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
            for (int r = 0; r < L; ++r) a[i * L + r] *= inv;
        }
    }
    if (rc == ORC_OK) memcpy(Z_out, a, sizeof(double) * (size_t)(n * dims[n_layers]));
    free(a);
    free(b);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* k-means (Definition 2 / Section III-C: "apply KMeans")                                */
/* ------------------------------------------------------------------------------------ */
static double sqdist64(const double* x, const double* y, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = x[k] - y[k];
        s += t * t;
    }
    return s;
}

/* The same squared distance taken in single precision, term by term in ascending k with
 * separately rounded subtract, multiply and add (no fused multiply-add).  Used only where
 * the k-means++ sampling decision is compared with a single-precision kernel. */
static float sqdist32(const double* x, const double* y, int d) {
    float s = 0.0f;
    for (int k = 0; k < d; ++k) {
        volatile float t = (float)x[k] - (float)y[k];
        volatile float t2 = t * t;
        s = s + t2;
    }
    return s;
}

static uint64_t mulhi64(uint64_t a, uint64_t b) {
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

static uint64_t kmpp_draw(uint64_t seed, int64_t t) {
    uint32_t x[4];
    philox_stream(seed, (uint32_t)t, (uint32_t)((uint64_t)t >> 32), 0u, ORC_STREAM_KMPP, x);
    return (uint64_t)x[0] | ((uint64_t)x[1] << 32);
}

/* k-means++ seeding (Arthur & Vassilvitskii 2007): the first seed uniform, every later seed
 * drawn with probability proportional to D^2, the squared distance to the nearest seed so
 * far.  D^2 is quantised to q_i = floor(D^2_i * 2^40) (exact integers, so the cumulative
 * sums are order-free); draw t = floor(r * sum q / 2^64) and take the smallest i whose
 * inclusive prefix sum exceeds t.  If every q_i is 0 the lowest-index point not yet chosen
 * is taken.  fp32_decision selects the single-precision D^2 (see sqdist32). */
int orc_kmeanspp(const double* Z, int64_t n, int d, int K, uint64_t seed, int fp32_decision, int64_t* seeds) {
    if (K < 1 || K > n) return ORC_EINVAL;
    double* D2 = (double*)malloc(sizeof(double) * (size_t)n);
    unsigned char* chosen = (unsigned char*)calloc((size_t)n, 1);
    if (!D2 || !chosen) { free(D2); free(chosen); return ORC_ENOMEM; }
    int64_t first = (int64_t)mulhi64(kmpp_draw(seed, 0), (uint64_t)n);
    seeds[0] = first;
    chosen[first] = 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        D2[i] = fp32_decision ? (double)sqdist32(Z + i * d, Z + first * d, d) : sqdist64(Z + i * d, Z + first * d, d);
    for (int t = 1; t < K; ++t) {
        uint64_t total = 0;   /* an exact integer sum: its value does not depend on the order */
#pragma omp parallel for schedule(static) reduction(+ : total)
        for (int64_t i = 0; i < n; ++i) total += (uint64_t)(D2[i] * 1099511627776.0);
        int64_t pick = -1;
        if (total == 0) {
            for (int64_t i = 0; i < n; ++i) if (!chosen[i]) { pick = i; break; }
        } else {
            uint64_t thr = mulhi64(kmpp_draw(seed, t), total);
            uint64_t prefix = 0;
            for (int64_t i = 0; i < n; ++i) {
                prefix += (uint64_t)(D2[i] * 1099511627776.0);
                if (prefix > thr) { pick = i; break; }
            }
        }
        seeds[t] = pick;
        chosen[pick] = 1;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double nd = fp32_decision ? (double)sqdist32(Z + i * d, Z + pick * d, d) : sqdist64(Z + i * d, Z + pick * d, d);
            if (nd < D2[i]) D2[i] = nd;
        }
    }
    free(D2);
    free(chosen);
    return ORC_OK;
}

/* Lloyd's iterations from the given centroids mu (K x d, updated in place).  Each pass
 * assigns every point to its nearest centroid (ties to the lowest index); the pass stops
 * the loop if no label changed, otherwise every non-empty cluster's centroid becomes the
 * mean of its points (an empty cluster keeps its centroid).  At most T passes; after the T-th
 * the centroids are left as they were, so mu holds the centroids of the final assignment.
 * Returns the number of assignment passes in *passes; labels get the last assignment.
 * If `objective` is not NULL, objective[p] = sum_i ||z_i - mu_{label_i}||^2 of pass p. */
int orc_lloyd(const double* Z, int64_t n, int d, int K, double* mu, int T, int32_t* labels, int* passes,
              double* objective) {
    int32_t* nl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    double* bestd = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (!nl || !bestd) { free(nl); free(bestd); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) labels[i] = -1;
    int p = 0;
    for (p = 1; p <= T; ++p) {
        int64_t changed = 0;
#pragma omp parallel for schedule(static) reduction(+ : changed)
        for (int64_t i = 0; i < n; ++i) {
            double best = 0.0;
            int bc = -1;
            for (int c = 0; c < K; ++c) {
                double dist = sqdist64(Z + i * d, mu + (int64_t)c * d, d);
                if (bc < 0 || dist < best) { best = dist; bc = c; }
            }
            nl[i] = bc;
            bestd[i] = best;
            if (bc != labels[i]) ++changed;
        }
        if (objective) {
            double obj = 0.0;   /* summed in index order */
            for (int64_t i = 0; i < n; ++i) obj += bestd[i];
            objective[p - 1] = obj;
        }
        if (changed == 0) break;
        for (int64_t i = 0; i < n; ++i) labels[i] = nl[i];
        if (p == T) break;   /* the returned centroids are those the final labels were assigned against */
        int rc = ORC_OK;
#pragma omp parallel
        {
        double* sum = (double*)malloc(sizeof(double) * (size_t)d);
        if (!sum) {
#pragma omp atomic write
            rc = ORC_ENOMEM;
        }
#pragma omp for schedule(dynamic, 1)
        for (int c = 0; c < K; ++c) {
            if (!sum) continue;
            int64_t cnt = 0;
            for (int k = 0; k < d; ++k) sum[k] = 0.0;
            for (int64_t i = 0; i < n; ++i) {   /* the members of c, in index order */
                if (labels[i] != c) continue;
                ++cnt;
                for (int k = 0; k < d; ++k) sum[k] += Z[i * d + k];
            }
            if (cnt > 0)
                for (int k = 0; k < d; ++k) mu[(int64_t)c * d + k] = sum[k] / (double)cnt;
        }
        free(sum);
        }
        if (rc != ORC_OK) { free(nl); free(bestd); return rc; }
    }
    *passes = p > T ? T : p;
    free(nl);
    free(bestd);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Scores: Eq. 1 (NCut), Eq. 3 (Mod) via Eq. 7 with U = V                               */
/* ------------------------------------------------------------------------------------ */
/* m_r = number of undirected edges with both ends in block r; vol_r = sum of degrees in r.
 * Mod = sum_r [m_r/e - (vol_r/2e)^2] = (2*(2e)*sum_r m_r - sum_r vol_r^2) / (2e)^2,
 * numerator and denominator exact integers, one FP64 division.
 * NCut = 1/2 sum_{r: vol_r > 0} cut_r / vol_r with cut_r = vol_r - 2 m_r, r ascending. */
int orc_score(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* labels, int K,
              int64_t* m, int64_t* vol, double* mod, double* ncut) {
    for (int r = 0; r < K; ++r) { m[r] = 0; vol[r] = 0; }
    for (int64_t i = 0; i < n; ++i) if (labels[i] < 0 || labels[i] >= K) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
        vol[labels[i]] += degree(row_ptr, i);
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int64_t j = col[p];
            if (i < j && labels[i] == labels[j]) m[labels[i]] += 1;
        }
    }
    int64_t two_e = row_ptr[n];
    __int128 msum = 0, vsq = 0;
    for (int r = 0; r < K; ++r) {
        msum += m[r];
        vsq += (__int128)vol[r] * vol[r];
    }
    __int128 num = 2 * (__int128)two_e * msum - vsq;
    __int128 den = (__int128)two_e * two_e;
    *mod = den > 0 ? (double)num / (double)den : 0.0;
    double s = 0.0;
    for (int r = 0; r < K; ++r)
        if (vol[r] > 0) s += (double)(vol[r] - 2 * m[r]) / (double)vol[r];
    *ncut = 0.5 * s;
    return ORC_OK;
}

/* Local modularity, Def. 5 / Eq. 7, for a partition of a node subset U of G:
 * LMod = sum_r [m_r/e_U - (mbar_r / 2e_U)^2], mbar_r the G-degree total of U_r and
 * 2e_U = sum_r mbar_r (the paper's definition of e inside Def. 5).  m_r counts edges of G
 * with both ends in U_r.  `in_u` marks U; labels are read only on U. */
int orc_local_modularity(int64_t n, const int64_t* row_ptr, const int32_t* col, const unsigned char* in_u,
                         const int32_t* labels, int K, double* lmod) {
    int64_t* m = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    int64_t* vb = (int64_t*)calloc((size_t)K, sizeof(int64_t));
    if (!m || !vb) { free(m); free(vb); return ORC_ENOMEM; }
    int64_t two_eu = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!in_u[i]) continue;
        int r = labels[i];
        if (r < 0 || r >= K) { free(m); free(vb); return ORC_EINVAL; }
        vb[r] += degree(row_ptr, i);
        two_eu += degree(row_ptr, i);
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int64_t j = col[p];
            if (i < j && in_u[j] && labels[j] == r) m[r] += 1;
        }
    }
    double s = 0.0;
    if (two_eu > 0) {
        double e = 0.5 * (double)two_eu;
        for (int r = 0; r < K; ++r) {
            double f = (double)vb[r] / (double)two_eu;
            s += (double)m[r] / e - f * f;
        }
    }
    *lmod = s;
    free(m);
    free(vb);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Model selection over candidate K                                                      */
/* ------------------------------------------------------------------------------------ */
/* Coarse grid: G values kmin + round((kmax-kmin) * t / (G-1)), t = 0..G-1 (round half up),
 * duplicates dropped.  Returns the count. */
int orc_coarse_grid(int kmin, int kmax, int G, int* out) {
    int cnt = 0;
    for (int t = 0; t < G; ++t) {
        int64_t num = 2 * (int64_t)(kmax - kmin) * t + (G - 1);
        int k = kmin + (int)(num / (2 * (int64_t)(G - 1)));
        if (cnt == 0 || out[cnt - 1] != k) out[cnt++] = k;
    }
    return cnt;
}

/* Refined grid between the neighbours of the best coarse value: lo + round((hi-lo)*t/(G+1)),
 * t = 1..G, keeping values not in `done` (n_done entries) and not already listed. */
int orc_refine_grid(int lo, int hi, int G, const int* done, int n_done, int* out) {
    int cnt = 0;
    for (int t = 1; t <= G; ++t) {
        int64_t num = 2 * (int64_t)(hi - lo) * t + (G + 1);
        int k = lo + (int)(num / (2 * (int64_t)(G + 1)));
        int seen = 0;
        for (int u = 0; u < n_done; ++u) if (done[u] == k) seen = 1;
        for (int u = 0; u < cnt; ++u) if (out[u] == k) seen = 1;
        if (!seen) out[cnt++] = k;
    }
    return cnt;
}

static int better(int criterion, double mod_a, double ncut_a, int k_a, double mod_b, double ncut_b, int k_b) {
    /* is candidate a better than candidate b?  exact ties go to the smaller K */
    if (criterion == ORC_CRIT_NCUT) {
        if (ncut_a != ncut_b) return ncut_a < ncut_b;
    } else {
        if (mod_a != mod_b) return mod_a > mod_b;
    }
    return k_a < k_b;
}

/* One candidate: the first K k-means++ seeds as initial centroids, Lloyd, score. */
static int eval_candidate(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* Z, int d, int K,
                          const int64_t* seeds, int T, int32_t* labels, double* mod, double* ncut, int* passes) {
    double* mu = (double*)malloc(sizeof(double) * (size_t)K * (size_t)d);
    int64_t* m = (int64_t*)malloc(sizeof(int64_t) * (size_t)K);
    int64_t* vol = (int64_t*)malloc(sizeof(int64_t) * (size_t)K);
    if (!mu || !m || !vol) { free(mu); free(m); free(vol); return ORC_ENOMEM; }
    for (int c = 0; c < K; ++c) memcpy(mu + (int64_t)c * d, Z + seeds[c] * d, sizeof(double) * (size_t)d);
    int rc = orc_lloyd(Z, n, d, K, mu, T, labels, passes, NULL);
    if (rc == ORC_OK) rc = orc_score(n, row_ptr, col, labels, K, m, vol, mod, ncut);
    free(mu); free(m); free(vol);
    return rc;
}

/* Model selection: candidates K in [kmin, kmax] (flat when grid == 0, else a coarse grid
 * of `grid` values and one refined grid of `grid` values around the best), one k-means++
 * run for K = kmax shared by all candidates (candidate K starts from the first K seeds),
 * Lloyd for each, the best by the criterion (modularity by default).  seed_fp32 selects the
 * single-precision D^2 for the seeding decisions (see orc_kmeanspp).
 * Outputs: labels (n) of the best; cand_k / cand_mod / cand_ncut / cand_passes for every
 * evaluated candidate in evaluation order (arrays of capacity max_cand); returns the
 * number evaluated in *n_cand and the chosen K in *k_best. */
int orc_select(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* Z, int d, int kmin, int kmax,
               int grid, int T, uint64_t seed, int criterion, int seed_fp32, int max_cand, int32_t* labels,
               int* k_best, int* n_cand, int* cand_k, double* cand_mod, double* cand_ncut, int* cand_passes) {
    if (kmax > n) kmax = (int)n;
    if (kmin < 1 || kmin > kmax) return ORC_EINVAL;
    int64_t* seeds = (int64_t*)malloc(sizeof(int64_t) * (size_t)kmax);
    int32_t* lab = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int* list = (int*)malloc(sizeof(int) * (size_t)(kmax - kmin + 2 + 2 * grid));
    if (!seeds || !lab || !list) { free(seeds); free(lab); free(list); return ORC_ENOMEM; }
    int rc = orc_kmeanspp(Z, n, d, kmax, seed, seed_fp32, seeds);
    int count = 0, best = -1;
    int stages = grid > 0 ? 2 : 1;
    for (int stage = 0; stage < stages && rc == ORC_OK; ++stage) {
        int nl = 0;
        if (grid == 0) {
            for (int k = kmin; k <= kmax; ++k) list[nl++] = k;
        } else if (stage == 0) {
            nl = orc_coarse_grid(kmin, kmax, grid, list);
        } else {
            /* neighbours of the best coarse value inside the coarse list */
            int ncoarse = count, jb = best;
            int lo = cand_k[jb > 0 ? jb - 1 : 0];
            int hi = cand_k[jb < ncoarse - 1 ? jb + 1 : ncoarse - 1];
            nl = orc_refine_grid(lo, hi, grid, cand_k, count, list);
        }
        for (int u = 0; u < nl && rc == ORC_OK; ++u) {
            if (count >= max_cand) { rc = ORC_EINVAL; break; }
            int K = list[u];
            double mod, ncut;
            int passes;
            rc = eval_candidate(n, row_ptr, col, Z, d, K, seeds, T, lab, &mod, &ncut, &passes);
            if (rc) break;
            cand_k[count] = K; cand_mod[count] = mod; cand_ncut[count] = ncut; cand_passes[count] = passes;
            if (best < 0 || better(criterion, mod, ncut, K, cand_mod[best], cand_ncut[best], cand_k[best])) {
                best = count;
                memcpy(labels, lab, sizeof(int32_t) * (size_t)n);
            }
            ++count;
        }
    }
    *n_cand = count;
    *k_best = best >= 0 ? cand_k[best] : 0;
    free(seeds); free(lab); free(list);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 2 (Section IV): graphs from the degree-corrected SBM of Definition 1,       */
/* A_ij ~ Pois(lambda_ij), lambda_ij = theta_i theta_j Omega_{c_i c_j}.                  */
/*                                                                                       */
/* Readings (the paper is silent on these):                                              */
/*   - Undirected, no self loops: block pairs r <= s; for r = s only the entries i < j   */
/*     (the upper triangle without the diagonal).                                        */
/*   - C_r lists the nodes of block r in ascending index order; the virtual table of     */
/*     (r, s) is row-major over (position in C_r, position in C_s), upper triangle rows  */
/*     for r = s (row a holds b = a+1 .. n_r-1).                                         */
/*   - Each table is cut into segments of `seg` consecutive entries (2^16 in the        */
/*     library) and the loop of Algorithm 2 runs on each segment on its own.  The        */
/*     entries are independent, so                                                        */
/*     the cut leaves the distribution unchanged; it fixes which draws each segment      */
/*     uses: draw j of global segment g comes from Philox counter (g_lo, g_hi, j,        */
/*     "Sbm2"), words 0-1 the skip uniform, words 2-3 the weight uniform.               */
/*   - The skip: p = (x >> 11 + 1) 2^-53 in (0, 1] from the 64-bit word x = w0 | w1 << 32,*/
/*     E = -ln p; with F(t) the sum of lambda over the entries before linear index t,    */
/*     the next nonzero entry is the smallest t >= m with F(t+1) > F(m) + E (i.e.        */
/*     p > exp(-RangeSum(m, t))), found by binary search on [m, segment end); none if    */
/*     F(segment end) <= F(m) + E.                                                        */
/*   - F from per-block prefix sums of theta, summed left to right:                      */
/*       r < s:  F(a, b) = om (Pre_r[a] Tot_s) + om (theta_a Pre_s[b])                  */
/*       r = s:  F(a, b) = om Tri_r[a] + om (theta_a (Pre_r[b] - Pre_r[a+1])),            */
/*               Tri_r[a] = sum_{a' < a} theta_a' (Tot_r - Pre_r[a'+1])                   */
/*     (a, b) being the table entry at linear index t, or the start of the next row.     */
/*   - The weight: A_ij ~ Pois(lambda) given A_ij >= 1 by inversion from k = 1 with the  */
/*     uniform u = (y >> 11) 2^-53 of words 2-3: P(1 | >= 1) = lambda / expm1(lambda),   */
/*     each next term times lambda / k (exact for lambda <= 700; at most 2^20 steps).    */
/*   The output graph is the support of A (each nonzero entry one edge, weight kept     */
/*   separately), so multi-edges collapse to one edge.                                   */
/* ------------------------------------------------------------------------------------ */
#define ORC_STREAM_SBM 0x53626d32u      /* "Sbm2" */

typedef struct {
    int r, s;
    int64_t nr, ns;
    const int32_t* nodes_r;
    const int32_t* nodes_s;
    const double* th_r;   /* theta in C_r order */
    const double* th_s;
    const double* pre_r;
    const double* pre_s;
    const double* tri_r;
    double tot_s, om;
} SbmPair;

static int64_t sbm_tri_row_start(int64_t n, int64_t a) { return a * n - a * (a + 1) / 2; }

/* The table entry (a, b) at linear index t (t may equal the table size: the end). */
static void sbm_entry(const SbmPair* P, int64_t t, int64_t* a, int64_t* b) {
    if (P->r != P->s) {
        *a = t / P->ns;
        *b = t % P->ns;
        return;
    }
    int64_t n = P->nr;
    int64_t size = n * (n - 1) / 2;
    if (t >= size) { *a = n - 1; *b = n; return; }   /* the end: after the last row */
    double q = (double)(2 * n - 1);
    int64_t r = (int64_t)((q - sqrt(q * q - 8.0 * (double)t)) / 2.0);
    if (r < 0) r = 0;
    if (r > n - 2) r = n - 2;
    while (r > 0 && sbm_tri_row_start(n, r) > t) --r;
    while (r + 1 <= n - 2 && sbm_tri_row_start(n, r + 1) <= t) ++r;
    *a = r;
    *b = r + 1 + (t - sbm_tri_row_start(n, r));
}

static double sbm_F(const SbmPair* P, int64_t t) {
    int64_t a, b;
    sbm_entry(P, t, &a, &b);
    if (P->r != P->s) {
        if (a >= P->nr) return P->om * (P->pre_r[P->nr] * P->tot_s);
        double rowpart = P->om * (P->pre_r[a] * P->tot_s);
        double colpart = P->om * (P->th_r[a] * P->pre_s[b]);
        return rowpart + colpart;
    }
    double rowpart = P->om * P->tri_r[a];
    double colpart = P->om * (P->th_r[a] * (P->pre_r[b] - P->pre_r[a + 1]));
    return rowpart + colpart;
}

static int sbm_weight(double lam, uint64_t y) {
    double u = (double)(y >> 11) * (1.0 / 9007199254740992.0);
    double term = lam / expm1(lam);
    double c = term;
    int k = 1;
    while (u >= c && k < (1 << 20)) {
        ++k;
        term = term * (lam / (double)k);
        c = c + term;
    }
    return k;
}

/* n nodes in K blocks (block[i] in [0, K)), theta[n] > 0, omega[K*K] row-major (entries
 * with r <= s read), segments of `seg` table entries.  Writes at most max_edges edges (src, dst, weight; any may be NULL
 * to only count) in the order (pair, segment, draw) and the count in *m_out. */
int orc_sbm_sample(int64_t n, int K, const int32_t* block, const double* theta, const double* omega, uint64_t seed,
                   int64_t seg, int64_t max_edges, int32_t* src, int32_t* dst, int32_t* weight, int64_t* m_out) {
    if (n < 0 || K < 1 || seg < 1) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if (block[i] < 0 || block[i] >= K || !(theta[i] >= 0.0)) return ORC_EINVAL;
    int64_t* boff = (int64_t*)calloc((size_t)K + 1, sizeof(int64_t));
    int32_t* nodes = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    double* th = (double*)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double* pre = (double*)malloc(sizeof(double) * (size_t)(n + K));
    double* tri = (double*)malloc(sizeof(double) * (size_t)(n + K));
    if (!boff || !nodes || !th || !pre || !tri) {
        free(boff); free(nodes); free(th); free(pre); free(tri);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) boff[block[i] + 1]++;
    for (int r = 0; r < K; ++r) boff[r + 1] += boff[r];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)K);
        if (!fill) { free(boff); free(nodes); free(th); free(pre); free(tri); return ORC_ENOMEM; }
        for (int r = 0; r < K; ++r) fill[r] = boff[r];
        for (int64_t i = 0; i < n; ++i) {   /* ascending node order inside each block */
            int64_t q = fill[block[i]]++;
            nodes[q] = (int32_t)i;
            th[q] = theta[i];
        }
        free(fill);
    }
    /* per block: Pre (n_r + 1 entries) and Tri (n_r + 1 entries) at offset boff[r] + r */
    for (int r = 0; r < K; ++r) {
        int64_t o = boff[r], nr = boff[r + 1] - boff[r];
        double* P = pre + o + r;
        double* T = tri + o + r;
        P[0] = 0.0;
        for (int64_t k = 0; k < nr; ++k) P[k + 1] = P[k] + th[o + k];
        double tot = P[nr];
        T[0] = 0.0;
        for (int64_t a = 0; a < nr; ++a) T[a + 1] = T[a] + th[o + a] * (tot - P[a + 1]);
    }
    int64_t m = 0, g = 0;
    int rc = ORC_OK;
    for (int r = 0; r < K && rc == ORC_OK; ++r) {
        for (int s = r; s < K && rc == ORC_OK; ++s) {
            SbmPair Pp;
            Pp.r = r; Pp.s = s;
            Pp.nr = boff[r + 1] - boff[r];
            Pp.ns = boff[s + 1] - boff[s];
            Pp.nodes_r = nodes + boff[r];
            Pp.nodes_s = nodes + boff[s];
            Pp.th_r = th + boff[r];
            Pp.th_s = th + boff[s];
            Pp.pre_r = pre + boff[r] + r;
            Pp.pre_s = pre + boff[s] + s;
            Pp.tri_r = tri + boff[r] + r;
            Pp.tot_s = Pp.pre_s[Pp.ns];
            Pp.om = omega[(int64_t)r * K + s];
            int64_t size = r != s ? Pp.nr * Pp.ns : Pp.nr * (Pp.nr - 1) / 2;
            int64_t nseg = (size + seg - 1) / seg;
            for (int64_t sg = 0; sg < nseg; ++sg, ++g) {
                int64_t t0 = sg * seg;
                int64_t t1 = t0 + seg < size ? t0 + seg : size;
                int64_t mm = t0;
                uint32_t j = 0;
                double Fend = sbm_F(&Pp, t1);
                while (mm < t1) {
                    uint32_t x[4];
                    philox_stream(seed, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), j, ORC_STREAM_SBM, x);
                    ++j;
                    uint64_t w01 = (uint64_t)x[0] | ((uint64_t)x[1] << 32);
                    uint64_t w23 = (uint64_t)x[2] | ((uint64_t)x[3] << 32);
                    double p = (double)((w01 >> 11) + 1) * (1.0 / 9007199254740992.0);
                    double V = sbm_F(&Pp, mm) + (-log(p));
                    if (!(Fend > V)) break;
                    int64_t lo = mm, hi = t1 - 1;
                    while (lo < hi) {
                        int64_t mid = lo + (hi - lo) / 2;
                        if (sbm_F(&Pp, mid + 1) > V) hi = mid;
                        else lo = mid + 1;
                    }
                    int64_t a, b;
                    sbm_entry(&Pp, lo, &a, &b);
                    if (m < max_edges) {
                        double lam = Pp.om * (Pp.th_r[a] * Pp.th_s[b]);
                        if (src) src[m] = Pp.nodes_r[a];
                        if (dst) dst[m] = Pp.nodes_s[b];
                        if (weight) weight[m] = sbm_weight(lam, w23);
                    } else if (src || dst || weight) {
                        rc = ORC_ENOMEM;
                        break;
                    }
                    ++m;
                    mm = lo + 1;
                }
            }
        }
    }
    *m_out = m;
    free(boff); free(nodes); free(th); free(pre); free(tri);
    return rc;
}

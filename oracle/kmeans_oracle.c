/*
 * kmeans_oracle.c -- plain, slow, FP64 CPU oracle for the k-means hot path of
 * "Solving k-means on High-dimensional Big Data" (Kappmeier, Schmidt, Schmidt).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline / reference arm may load this library.  It shares no
 * code, header, table or helper with the CUDA library; the two meet only
 * through the seeded input arrays.
 *
 * Every function computes its quantity from the definition, in double
 * precision, with plain loops in the order the paper states the step:
 *
 *   orc_row_norms   ||x_i||^2                                  (Section 2.1, CF sum of squares)
 *   orc_assign      nearest center by full scan                (Section 1, Lloyd's assignment step)
 *   orc_update      clustering features and centroids          (Section 1 update step; Section 2 mu(P);
 *                                                               Section 2.1 CF and its cost identity)
 *   orc_cost        sum_i w_i min_j ||x_i - c_j||^2            (Section 1, k-means objective)
 *   orc_cost_cf     cost of a labelled set from its CFs        (Section 2.1 identity)
 *   orc_pp_pick     one D^2 draw given D^2 and u               (Section 1, k-means++)
 *   orc_seed_pp     k-means++ seeding                          (Section 1, k-means++)
 *   orc_lloyd       seeding-free Lloyd iterations              (Section 1)
 *   orc_project     Y = X V and the lift Y V^T                 (Section 2.2, best-fit subspace projection)
 *   orc_quant_bf16  round-to-nearest-even to bfloat16          (precision form; no paper counterpart)
 *   orc_quant_e4m3  E4M3 with one power-of-two scale per block (precision form; no paper counterpart)
 *
 * Readings of the paper that these functions fix (where it is silent):
 *   - points are rows of a row-major n x d matrix;
 *   - argmin ties go to the lowest center index;
 *   - an empty cluster keeps its previous center;
 *   - k-means++ draws its first center uniformly (proportional to w when weighted),
 *     every later center with probability proportional to w_i * D^2_i, taking the
 *     smallest i whose inclusive prefix sum exceeds u * total; if rounding leaves
 *     u * total >= the full sum, the last i with w_i * D^2_i > 0 is taken;
 *   - the projection is onto the linear span of V (no centering).
 *
 * Parity: every function is pinned by tests against closed forms, brute force,
 * independent library routines or invariants; none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_EDEGENERATE (-6)

static int g_threads = 1;

int orc_set_threads(int t) {
    g_threads = t < 1 ? 1 : t;
#ifdef _OPENMP
    omp_set_num_threads(g_threads);
    return g_threads;
#else
    return 1;
#endif
}

int orc_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* squared Euclidean distance of an FP32 point to an FP64 center, by direct differences */
static double sqdist(const float *x, const double *c, int64_t d) {
    double s = 0.0;
    for (int64_t t = 0; t < d; ++t) {
        double diff = (double)x[t] - c[t];
        s += diff * diff;
    }
    return s;
}

/* ||x_i||^2 for every row (Section 2.1: the sum-of-squares part of a clustering feature) */
int orc_row_norms(const float *X, int64_t n, int64_t d, double *out) {
    if (n < 0 || d < 1) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t t = 0; t < d; ++t) s += (double)X[i * d + t] * (double)X[i * d + t];
        out[i] = s;
    }
    return ORC_OK;
}

/*
 * Assignment step of Lloyd's algorithm (Section 1): every point goes to its
 * closest center.  Full scan over the k centers; ties to the lowest index.
 * d1[i] is the smallest squared distance, d2[i] the second smallest
 * (+inf when k == 1), both in FP64 by direct differences.
 */
int orc_assign(const float *X, int64_t n, int64_t d, const double *C, int64_t k,
               int32_t *labels, double *d1, double *d2) {
    if (n < 0 || d < 1 || k < 1) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double best = INFINITY, second = INFINITY;
        int64_t arg = 0;
        for (int64_t j = 0; j < k; ++j) {
            double dist = sqdist(X + i * d, C + j * d, d);
            if (dist < best) {
                second = best;
                best = dist;
                arg = j;
            } else if (dist < second) {
                second = dist;
            }
        }
        labels[i] = (int32_t)arg;
        if (d1) d1[i] = best;
        if (d2) d2[i] = second;
    }
    return ORC_OK;
}

/*
 * Update step (Section 1: replace each center by the centroid of its subset;
 * Section 2: mu(P) = sum x / |P|) computed through clustering features
 * (Section 2.1): N_j = sum w_i, S_j = sum w_i x_i, Q_j = sum w_i x_i^T x_i over
 * the points labelled j.  C_new[j] = S_j / N_j, or C_old[j] when N_j == 0.
 *
 * cost_old = cost(C_old, labels) and cost_new = cost(C_new, labels) are summed
 * directly over the points (sum_i w_i ||x_i - c_{l_i}||^2); orc_cost_cf gives the
 * same two numbers from the CFs.  w may be NULL (all weights 1).
 */
int orc_update(const float *X, int64_t n, int64_t d, const double *w, const int32_t *labels,
               int64_t k, const double *C_old, double *C_new, double *N, double *S, double *Q,
               double *cost_old, double *cost_new, int64_t *n_empty) {
    if (n < 0 || d < 1 || k < 1) return ORC_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if (labels[i] < 0 || labels[i] >= k) return ORC_EINVAL;
    memset(N, 0, sizeof(double) * k);
    memset(S, 0, sizeof(double) * k * d);
    memset(Q, 0, sizeof(double) * k);
    for (int64_t i = 0; i < n; ++i) {
        int64_t j = labels[i];
        double wi = w ? w[i] : 1.0;
        N[j] += wi;
        for (int64_t t = 0; t < d; ++t) {
            S[j * d + t] += wi * (double)X[i * d + t];
            Q[j] += wi * (double)X[i * d + t] * (double)X[i * d + t];
        }
    }
    int64_t empty = 0;
    for (int64_t j = 0; j < k; ++j) {
        if (N[j] == 0.0) {
            ++empty;
            for (int64_t t = 0; t < d; ++t) C_new[j * d + t] = C_old[j * d + t];
        } else {
            for (int64_t t = 0; t < d; ++t) C_new[j * d + t] = S[j * d + t] / N[j];
        }
    }
    if (n_empty) *n_empty = empty;
    double co = 0.0, cn = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t j = labels[i];
        double wi = w ? w[i] : 1.0;
        co += wi * sqdist(X + i * d, C_old + j * d, d);
        cn += wi * sqdist(X + i * d, C_new + j * d, d);
    }
    if (cost_old) *cost_old = co;
    if (cost_new) *cost_new = cn;
    return ORC_OK;
}

/* k-means objective (Section 1): sum over points of w_i * (squared distance to the closest center) */
int orc_cost(const float *X, int64_t n, int64_t d, const double *w, const double *C, int64_t k,
             double *cost) {
    if (n < 0 || d < 1 || k < 1) return ORC_EINVAL;
    double *per = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    if (!per) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double best = INFINITY;
        for (int64_t j = 0; j < k; ++j) {
            double dist = sqdist(X + i * d, C + j * d, d);
            if (dist < best) best = dist;
        }
        per[i] = (w ? w[i] : 1.0) * best;
    }
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += per[i];
    free(per);
    *cost = s;
    return ORC_OK;
}

/*
 * Cost of a labelled set against centers C from its clustering features
 * (Section 2.1): sum_{x in P} ||x - c||^2 = |P| ||mu(P) - c||^2 + sum ||x - mu(P)||^2,
 * written with the three CF sums as  Q_j - 2 c_j . S_j + N_j ||c_j||^2.
 */
int orc_cost_cf(const double *N, const double *S, const double *Q, const double *C, int64_t k,
                int64_t d, double *cost) {
    double s = 0.0;
    for (int64_t j = 0; j < k; ++j) {
        double cs = 0.0, cc = 0.0;
        for (int64_t t = 0; t < d; ++t) {
            cs += C[j * d + t] * S[j * d + t];
            cc += C[j * d + t] * C[j * d + t];
        }
        s += Q[j] - 2.0 * cs + N[j] * cc;
    }
    *cost = s;
    return ORC_OK;
}

/*
 * One k-means++ draw (Section 1): point i is chosen with probability
 * proportional to p_i = w_i * D2_i.  With the inclusive prefix sums
 * P_i = p_0 + ... + p_i (summed left to right) and t = u * P_{n-1}, the draw is
 * the smallest i with P_i > t; if rounding leaves t >= P_{n-1}, the last i with
 * p_i > 0.  Returns ORC_EDEGENERATE when every p_i is zero.
 */
int orc_pp_pick(const double *D2, const double *w, int64_t n, double u, int64_t *idx) {
    double total = 0.0;
    for (int64_t i = 0; i < n; ++i) total += (w ? w[i] : 1.0) * D2[i];
    if (!(total > 0.0)) return ORC_EDEGENERATE;
    double t = u * total;
    double run = 0.0;
    int64_t last_pos = -1;
    for (int64_t i = 0; i < n; ++i) {
        double p = (w ? w[i] : 1.0) * D2[i];
        run += p;
        if (p > 0.0) last_pos = i;
        if (run > t) {
            *idx = i;
            return ORC_OK;
        }
    }
    *idx = last_pos;
    return ORC_OK;
}

/*
 * k-means++ seeding (Section 1).  The first center is drawn uniformly
 * (index floor(u[0] * n)), or proportionally to w when weights are given (a
 * prefix search of u[0] * sum w).  Afterwards D2_i = min over chosen centers of
 * ||x_i - c||^2 and center j is drawn by orc_pp_pick with u[j].
 * idx_out receives the k chosen row indices, C_out (nullable) the k x d centers
 * (FP64 copies of the chosen rows), D2_out (nullable) the final D^2.
 * If fewer than k points have positive weighted D^2 the function stops and
 * returns ORC_EDEGENERATE with the centers chosen so far in idx_out.
 */
int orc_seed_pp(const float *X, int64_t n, int64_t d, const double *w, int64_t k,
                const double *u, int64_t *idx_out, double *C_out, double *D2_out) {
    if (n < 1 || d < 1 || k < 1 || k > n) return ORC_EINVAL;
    double *D2 = (double *)malloc(sizeof(double) * n);
    double *c = (double *)malloc(sizeof(double) * d);
    if (!D2 || !c) {
        free(D2);
        free(c);
        return ORC_EINVAL;
    }
    int64_t first;
    if (!w) {
        first = (int64_t)floor(u[0] * (double)n);
        if (first >= n) first = n - 1;
    } else {
        double ones_total = 0.0;
        for (int64_t i = 0; i < n; ++i) ones_total += w[i];
        double t = u[0] * ones_total, run = 0.0;
        first = -1;
        for (int64_t i = 0; i < n; ++i) {
            run += w[i];
            if (run > t) {
                first = i;
                break;
            }
        }
        if (first < 0) {
            for (int64_t i = n - 1; i >= 0; --i)
                if (w[i] > 0.0) {
                    first = i;
                    break;
                }
        }
    }
    int rc = ORC_OK;
    idx_out[0] = first;
    for (int64_t t = 0; t < d; ++t) c[t] = (double)X[first * d + t];
    if (C_out)
        for (int64_t t = 0; t < d; ++t) C_out[t] = c[t];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) D2[i] = sqdist(X + i * d, c, d);
    D2[first] = 0.0;
    for (int64_t j = 1; j < k; ++j) {
        int64_t pick;
        rc = orc_pp_pick(D2, w, n, u[j], &pick);
        if (rc != ORC_OK) break;
        idx_out[j] = pick;
        for (int64_t t = 0; t < d; ++t) c[t] = (double)X[pick * d + t];
        if (C_out)
            for (int64_t t = 0; t < d; ++t) C_out[j * d + t] = c[t];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double dist = sqdist(X + i * d, c, d);
            if (dist < D2[i]) D2[i] = dist;
        }
        D2[pick] = 0.0;
    }
    if (D2_out) memcpy(D2_out, D2, sizeof(double) * n);
    free(D2);
    free(c);
    return rc;
}

/*
 * Lloyd's algorithm (Section 1) from given centers C0 for `iters` iterations:
 * assign, then update.  cost_trace[2t] = cost(C_t, L_t), cost_trace[2t+1] =
 * cost(C_{t+1}, L_t), so a correct run is non-increasing along the trace.
 * conv_iter receives the first t >= 1 with L_t == L_{t-1} (-1 if none).
 */
int orc_lloyd(const float *X, int64_t n, int64_t d, const double *w, const double *C0, int64_t k,
              int64_t iters, double *C_out, int32_t *labels_out, double *cost_trace,
              int64_t *conv_iter) {
    if (n < 1 || d < 1 || k < 1 || iters < 0) return ORC_EINVAL;
    double *C = (double *)malloc(sizeof(double) * k * d);
    double *Cn = (double *)malloc(sizeof(double) * k * d);
    double *N = (double *)malloc(sizeof(double) * k);
    double *S = (double *)malloc(sizeof(double) * k * d);
    double *Q = (double *)malloc(sizeof(double) * k);
    int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!C || !Cn || !N || !S || !Q || !prev) return ORC_EINVAL;
    memcpy(C, C0, sizeof(double) * k * d);
    int64_t conv = -1;
    for (int64_t it = 0; it < iters; ++it) {
        orc_assign(X, n, d, C, k, labels_out, NULL, NULL);
        if (it > 0 && conv < 0 && memcmp(prev, labels_out, sizeof(int32_t) * n) == 0) conv = it;
        memcpy(prev, labels_out, sizeof(int32_t) * n);
        double co, cn;
        int64_t ne;
        orc_update(X, n, d, w, labels_out, k, C, Cn, N, S, Q, &co, &cn, &ne);
        if (cost_trace) {
            cost_trace[2 * it] = co;
            cost_trace[2 * it + 1] = cn;
        }
        memcpy(C, Cn, sizeof(double) * k * d);
    }
    memcpy(C_out, C, sizeof(double) * k * d);
    if (conv_iter) *conv_iter = conv;
    free(C);
    free(Cn);
    free(N);
    free(S);
    free(Q);
    free(prev);
    return ORC_OK;
}

/*
 * Projection onto the span of V (Section 2.2): with V a d x r matrix of
 * orthonormal columns (the top right singular vectors of the piece), the
 * r-dimensional coordinates are Y = X V and the paper's d-dimensional
 * A_l = U D_l V^T equals the lift Y V^T.  Y is n x r, lift (nullable) n x d.
 */
int orc_project(const float *X, int64_t n, int64_t d, const double *V, int64_t r, double *Y,
                double *lift) {
    if (n < 0 || d < 1 || r < 1) return ORC_EINVAL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t q = 0; q < r; ++q) {
            double s = 0.0;
            for (int64_t t = 0; t < d; ++t) s += (double)X[i * d + t] * V[t * r + q];
            Y[i * r + q] = s;
        }
        if (lift) {
            for (int64_t t = 0; t < d; ++t) {
                double s = 0.0;
                for (int64_t q = 0; q < r; ++q) s += Y[i * r + q] * V[t * r + q];
                lift[i * d + t] = s;
            }
        }
    }
    return ORC_OK;
}

/*
 * bfloat16 by its definition: keep the sign, the 8 exponent bits and the top
 * 7 fraction bits of the FP32 encoding, rounding the dropped 16 bits to
 * nearest, ties to even.  Output as the 16-bit pattern.  (NaN inputs are not
 * produced by the workloads; they map to a quiet NaN.)
 */
int orc_quant_bf16(const float *x, int64_t m, uint16_t *out) {
    for (int64_t i = 0; i < m; ++i) {
        uint32_t b;
        memcpy(&b, &x[i], 4);
        if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu)) {
            out[i] = (uint16_t)((b >> 16) | 0x40);
            continue;
        }
        uint32_t upper = b >> 16, lower = b & 0xffffu;
        if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1;
        out[i] = (uint16_t)upper;
    }
    return ORC_OK;
}

/* value of an E4M3 (fn variant: bias 7, no infinities, max 448) byte */
static double e4m3_value(uint8_t v) {
    int s = v >> 7, e = (v >> 3) & 15, m = v & 7;
    double mag = e == 0 ? ldexp((double)m, -9) : ldexp(1.0 + m / 8.0, e - 7);
    return s ? -mag : mag;
}

/*
 * E4M3 quantisation with one power-of-two scale per block of `block` elements
 * along each row: scale_b = 2^e with e the smallest integer such that
 * max_{t in b} |x_t| * 2^-e <= 448 (e = 0 for an all-zero block); each element is
 * x * 2^-e rounded to the nearest E4M3 value (ties to the even code), so that
 * x ~= scale * decode(q).  out is n x d bytes, scales n x ceil(d/block) FP32.
 */
int orc_quant_e4m3(const float *X, int64_t n, int64_t d, int64_t block, uint8_t *out,
                   float *scales) {
    if (block < 1) return ORC_EINVAL;
    int64_t nb = (d + block - 1) / block;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t b = 0; b < nb; ++b) {
            int64_t t0 = b * block, t1 = t0 + block < d ? t0 + block : d;
            double amax = 0.0;
            for (int64_t t = t0; t < t1; ++t) {
                double a = fabs((double)X[i * d + t]);
                if (a > amax) amax = a;
            }
            int e = 0;
            if (amax > 0.0) {
                e = -300;
                while (!(ldexp(amax, -e) <= 448.0)) ++e;
            }
            scales[i * nb + b] = (float)ldexp(1.0, e);
            for (int64_t t = t0; t < t1; ++t) {
                double v = ldexp((double)X[i * d + t], -e);
                double a = fabs(v);
                /* nearest magnitude code 0x00..0x7e (0x7f is NaN); ties -> even code */
                int best = 0;
                double bd = INFINITY;
                for (int code = 0; code < 0x7f; ++code) {
                    double diff = fabs(e4m3_value((uint8_t)code) - a);
                    if (diff < bd || (diff == bd && !(code & 1) && (best & 1))) {
                        bd = diff;
                        best = code;
                    }
                }
                if (signbit(v)) best |= 0x80;
                out[i * d + t] = (uint8_t)best;
            }
        }
    }
    return ORC_OK;
}

double orc_e4m3_decode(uint8_t v) { return e4m3_value(v); }

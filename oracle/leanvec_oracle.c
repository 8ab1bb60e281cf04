/*
 * CPU oracle for the LeanVec search path -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised restatement of what the paper
 * (LeanVec, arXiv 2312.16335) defines for the search path, written so that a
 * reader can check each function against the paper by eye:
 *
 *   - LVQ encode / decode (LVQ is cited in Sec. 2 for quant(.); its
 *     definition is the per-vector scalar quantiser of the LVQ paper).
 *   - primary / secondary inner products (Eq. 1, "Search" paragraph of Sec. 2).
 *   - best-first beam search ("greedy traversal with backtracking", App. D)
 *     followed by the rerank with secondary vectors (Sec. 2, "Search").
 *   - exact brute-force top-k (the definition of the search problem, Sec. 2).
 *   - RobustPrune and the batch-synchronous Vamana build (App. A, App. D).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library. It shares no code, header or helper with the CUDA library.
 *
 * Arithmetic: scores are FP64 except the build score, which is a fixed
 * sequence of FP32 operations on exact integer sums (so that a graph built
 * anywhere is reproducible bit for bit).  Compile with -ffp-contract=off.
 *
 * Metrics: inner product (the paper's setting), or squared Euclidean distance
 * ranked through the identity -||q - x||^2 = 2 <q, x> - ||x||^2 - ||q||^2 (the
 * query's norm is a per-query constant): the "L2 score" of x is 2 <q, x> - ||x||^2,
 * with <q, x> approximated exactly as for the inner product (Eq. 1) and ||x||^2
 * the squared norm of the original vector, kept per record.
 *
 * Pins: the paper prints no worked example for these functions; each is pinned
 * against something other than itself -- closed forms, invariants, special
 * cases that reduce to a textbook routine, brute force on tiny inputs and an
 * independent sequential replay -- in tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* LVQ: v = y - mean; l = min v; u = max v; delta = (u-l)/(2^b-1);      */
/* code = clamp(floor((v-l)/delta + 0.5), 0, 2^b-1); decode l + delta*c */
/* ------------------------------------------------------------------ */
int orc_lvq_encode(const float *Y, int64_t n, int dim, const float *mean, int bits,
                   uint8_t *codes, float *delta, float *lower)
{
    if (bits < 1 || bits > 8 || dim <= 0) return -1;
    const float levels = (float)((1 << bits) - 1);
    float *v = (float *)malloc(sizeof(float) * (size_t)dim);
    if (!v) return -2;
    for (int64_t i = 0; i < n; ++i) {
        const float *y = Y + i * (int64_t)dim;
        for (int j = 0; j < dim; ++j) v[j] = y[j] - mean[j];
        float lo = v[0], hi = v[0];
        for (int j = 1; j < dim; ++j) {
            if (v[j] < lo) lo = v[j];
            if (v[j] > hi) hi = v[j];
        }
        float dl = (hi - lo) / levels;
        delta[i] = dl;
        lower[i] = lo;
        uint8_t *c = codes + i * (int64_t)dim;
        for (int j = 0; j < dim; ++j) {
            if (dl > 0.0f) {
                float t = (v[j] - lo) / dl;
                float f = floorf(t + 0.5f);
                if (f < 0.0f) f = 0.0f;
                if (f > levels) f = levels;
                c[j] = (uint8_t)f;
            } else {
                c[j] = 0;
            }
        }
    }
    free(v);
    return 0;
}

/* decoded vector in FP64: mean_j + l + delta * c_j */
void orc_lvq_decode(const uint8_t *codes, const float *delta, const float *lower,
                    const float *mean, int64_t n, int dim, double *out)
{
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < dim; ++j)
            out[i * dim + j] = (double)mean[j] + (double)lower[i] +
                               (double)delta[i] * (double)codes[i * (int64_t)dim + j];
}

/* ------------------------------------------------------------------ */
/* Stores: what a database record decodes to.                          */
/* ------------------------------------------------------------------ */
typedef struct {
    int kind;             /* 0 = LVQ codes, 1 = raw fp32 vectors */
    int dim;
    const uint8_t *codes; /* n x dim, one code per byte */
    const float *delta;
    const float *lower;
    const float *mean;    /* dim */
    const float *vecs;    /* kind 1: n x dim */
    int metric;           /* 0 = inner product, 1 = L2 score 2 <q, x> - ||x||^2 */
    const float *sqnorm;  /* n: ||x_i||^2 of the original vectors (L2; kind 1 may pass NULL) */
} orc_store;

/* <q, decode(x_i)> in FP64 (decode first, then the plain dot product); for the
 * L2 metric 2 <q, decode(x_i)> - ||x_i||^2 (||x_i||^2 from sqnorm, or for raw
 * vectors without sqnorm the FP64 sum of squares). */
static double store_score(const orc_store *s, const double *q, int64_t i)
{
    double acc = 0.0, nrm = 0.0;
    if (s->kind == 0) {
        const uint8_t *c = s->codes + i * (int64_t)s->dim;
        double l = s->lower[i], dl = s->delta[i];
        for (int j = 0; j < s->dim; ++j)
            acc += q[j] * ((double)s->mean[j] + l + dl * (double)c[j]);
    } else {
        const float *x = s->vecs + i * (int64_t)s->dim;
        for (int j = 0; j < s->dim; ++j) {
            acc += q[j] * (double)x[j];
            nrm += (double)x[j] * (double)x[j];
        }
    }
    if (!s->metric) return acc;
    return 2.0 * acc - (s->sqnorm ? (double)s->sqnorm[i] : nrm);
}

/* ------------------------------------------------------------------ */
/* Build score: <y_a, y_b> of two decoded primaries, with the mean held  */
/* in 2^-20 fixed point, evaluated as exact integer sums combined by a   */
/* fixed sequence of FP32 operations (no fused multiply-add).           */
/*   y_j = mu_j + l + delta c_j, mu_j = mui_j * 2^-20                    */
/*   <y_a,y_b> = sum mu^2 + (G_a + G_b) + d l_a l_b                      */
/*             + (l_b H_a + l_a H_b) + delta_a delta_b P_ab              */
/*   G = l*sum(mu) + delta*sum(mu c), H = delta * sum(c), P = sum c_a c_b */
/* ------------------------------------------------------------------ */
typedef struct {
    int dim;
    const uint8_t *codes;
    const float *delta;
    const float *lower;
    float *G;      /* n, filled by orc_build_prepare */
    float *H;      /* n */
    const float *N; /* L2 metric: n self scores <y_i, y_i> (same arithmetic); NULL = inner product */
    float mu2;     /* sum mu^2 as float */
} orc_bstore;

static const double FIX = 1048576.0; /* 2^20 */

static float bscore_ip(const orc_bstore *b, int64_t a, int64_t c);

/* G, H, mu2 of the build score; N (nullable): the self scores <y_i, y_i> the L2 build
 * score needs. */
int orc_build_prepare(const uint8_t *codes, const float *delta, const float *lower,
                      const float *mean, int64_t n, int dim, float *G, float *H, float *N, float *mu2_out)
{
    int32_t *mui = (int32_t *)malloc(sizeof(int32_t) * (size_t)dim);
    if (!mui) return -2;
    int64_t s_mu = 0, s_mu2 = 0;
    for (int j = 0; j < dim; ++j) {
        if (!(fabsf(mean[j]) < 8.0f)) { free(mui); return -1; }
        mui[j] = (int32_t)llrint((double)mean[j] * FIX);
        s_mu += mui[j];
        s_mu2 += (int64_t)mui[j] * (int64_t)mui[j];
    }
    const float MU1 = (float)s_mu * (float)(1.0 / FIX);
    *mu2_out = (float)s_mu2 * (float)(1.0 / (FIX * FIX));
    for (int64_t i = 0; i < n; ++i) {
        const uint8_t *c = codes + i * (int64_t)dim;
        int64_t m = 0, s = 0;
        for (int j = 0; j < dim; ++j) {
            m += (int64_t)mui[j] * (int64_t)c[j];
            s += c[j];
        }
        float mf = (float)m * (float)(1.0 / FIX);
        float t1 = lower[i] * MU1;
        float t2 = delta[i] * mf;
        G[i] = t1 + t2;
        H[i] = delta[i] * (float)s;
    }
    free(mui);
    if (N) {
        orc_bstore bs = {dim, codes, delta, lower, G, H, NULL, *mu2_out};
        for (int64_t i = 0; i < n; ++i) N[i] = bscore_ip(&bs, i, i);
    }
    return 0;
}

static float bscore_ip(const orc_bstore *b, int64_t a, int64_t c)
{
    const uint8_t *ca = b->codes + a * (int64_t)b->dim;
    const uint8_t *cc = b->codes + c * (int64_t)b->dim;
    int32_t P = 0;
    for (int j = 0; j < b->dim; ++j) P += (int32_t)ca[j] * (int32_t)cc[j];
    float t1 = b->G[a] + b->G[c];
    float ll = b->lower[a] * b->lower[c];
    float t2 = (float)b->dim * ll;
    float h1 = b->lower[c] * b->H[a];
    float h2 = b->lower[a] * b->H[c];
    float t3 = h1 + h2;
    float dd = b->delta[a] * b->delta[c];
    float t4 = dd * (float)P;
    float s = b->mu2 + t1;
    s = s + t2;
    s = s + t3;
    s = s + t4;
    return s;
}

/* inner product: <y_a, y_c>; L2: -||y_a - y_c||^2 = 2 <y_a, y_c> - (N_a + N_c) in FP32
 * (the sum of the two self scores first, so that the score is symmetric bit for bit) */
static float bscore(const orc_bstore *b, int64_t a, int64_t c)
{
    const float ip = bscore_ip(b, a, c);
    if (!b->N) return ip;
    const float nn = b->N[a] + b->N[c];
    return 2.0f * ip - nn;
}

float orc_build_score(const uint8_t *codes, const float *delta, const float *lower,
                      const float *G, const float *H, const float *N, float mu2, int dim, int64_t a, int64_t b)
{
    orc_bstore bs = {dim, codes, delta, lower, (float *)G, (float *)H, N, mu2};
    return bscore(&bs, a, b);
}

/* ------------------------------------------------------------------ */
/* Candidate list: sorted by (score desc, id asc), capacity L.          */
/* ------------------------------------------------------------------ */
typedef struct { double s; int32_t id; int32_t expanded; } cand_t;

/* true when (sa,ia) ranks before (sb,ib) */
static int better(double sa, int32_t ia, double sb, int32_t ib)
{
    return sa > sb || (sa == sb && ia < ib);
}

static void cand_insert(cand_t *C, int *size, int L, double s, int32_t id)
{
    int n = *size;
    if (n == L && !better(s, id, C[n - 1].s, C[n - 1].id)) return;
    int pos = n;
    while (pos > 0 && better(s, id, C[pos - 1].s, C[pos - 1].id)) pos--;
    int last = (n == L) ? n - 1 : n;
    for (int t = last; t > pos; --t) C[t] = C[t - 1];
    C[pos].s = s; C[pos].id = id; C[pos].expanded = 0;
    if (n < L) *size = n + 1;
}

typedef struct {
    /* query-mode scorer */
    const orc_store *store;
    const double *q;
    /* build-mode scorer (store == NULL) */
    const orc_bstore *bs;
    int64_t qnode;
} scorer_t;

static double score_of(const scorer_t *sc, int64_t u)
{
    if (sc->store) return store_score(sc->store, sc->q, u);
    return (double)bscore(sc->bs, sc->qnode, u);
}

/* Best-first beam search.  C = {entry}; repeatedly take the `width` best
 * unexpanded members of C (fewer if fewer are left), mark them expanded and, parent
 * by parent in rank order and neighbour by neighbour in adjacency order, score each
 * not-yet-visited neighbour, keeping the best L of everything scored.  width = 1 is
 * the classic one-node-at-a-time traversal.  Stops when every member of C is
 * expanded or after max_hops expansions (max_hops <= 0: no limit; a round is cut
 * to the expansions left).  visited is an n-sized stamp array owned by the caller;
 * stamp must be fresh for this call.  Returns |C| and writes C. */
static int beam_search(const scorer_t *sc, const int32_t *graph, int R, int64_t n,
                       int32_t entry, int L, int max_hops, int width, uint32_t *visited, uint32_t stamp,
                       cand_t *C, int64_t *hops_out, int64_t *scored_out)
{
    int size = 0;
    int64_t hops = 0, scored = 1;
    int32_t par[64];
    if (width < 1) width = 1;
    if (width > 64) width = 64;
    visited[entry] = stamp;
    cand_insert(C, &size, L, score_of(sc, entry), entry);
    for (;;) {
        int np = 0;
        for (int i = 0; i < size && np < width; ++i) {
            if (C[i].expanded) continue;
            if (max_hops > 0 && hops + np >= max_hops) break;
            par[np++] = C[i].id;
        }
        if (np == 0) break;
        for (int t = 0; t < np; ++t)
            for (int i = 0; i < size; ++i)
                if (C[i].id == par[t]) C[i].expanded = 1;
        hops += np;
        for (int t = 0; t < np; ++t) {
            int32_t p = par[t];
            for (int j = 0; j < R; ++j) {
                int32_t u = graph[(int64_t)p * R + j];
                if (u < 0 || u >= n) continue;
                if (visited[u] == stamp) continue;
                visited[u] = stamp;
                scored++;
                cand_insert(C, &size, L, score_of(sc, u), u);
            }
        }
    }
    if (hops_out) *hops_out = hops;
    if (scored_out) *scored_out = scored;
    return size;
}

/*
 * Search + rerank for m queries (Sec. 2 "Search"), search width `width`:
 *   primary:   qp (m x dp, FP64 already projected: A q) scored against prim
 *   secondary: qs (m x ds, FP64 unreduced q)      scored against sec
 * Candidates are the top min(r, |C|) of the beam; they are rescored with the
 * secondary store and the best k returned (ties -> smaller id), padded with
 * id -1 / score -inf.  rerank r <= 0 or sec == NULL: return the top k of the
 * beam with primary scores.  beam_ids/beam_scores (nullable): m x L.
 */
int orc_search(const orc_store *prim, const orc_store *sec, const double *qp, const double *qs,
               int64_t m, const int32_t *graph, int64_t n, int R, int32_t entry,
               const int32_t *kLrh /* m x 4: k, L, r, max_hops */,
               int ldo, int32_t *ids, double *scores,
               int ldb, int32_t *beam_ids, double *beam_scores,
               int64_t *hops, int64_t *scored, int width, int nthreads)
{
    int Lmax = 1;
    for (int64_t i = 0; i < m; ++i) if (kLrh[4 * i + 1] > Lmax) Lmax = kLrh[4 * i + 1];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int err = 0;
#pragma omp parallel
    {
        uint32_t *visited = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
        cand_t *C = (cand_t *)malloc(sizeof(cand_t) * (size_t)(Lmax + 1));
        cand_t *R2 = (cand_t *)malloc(sizeof(cand_t) * (size_t)(Lmax + 1));
        uint32_t stamp = 0;
        if (!visited || !C || !R2) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t qi = 0; qi < m; ++qi) {
                int k = kLrh[4 * qi], L = kLrh[4 * qi + 1], r = kLrh[4 * qi + 2], mh = kLrh[4 * qi + 3];
                stamp++;
                if (stamp == 0) { memset(visited, 0, sizeof(uint32_t) * (size_t)n); stamp = 1; }
                scorer_t sc = {prim, qp + qi * (int64_t)prim->dim, NULL, 0};
                int64_t h = 0, sd = 0;
                int size = beam_search(&sc, graph, R, n, entry, L, mh, width, visited, stamp, C, &h, &sd);
                if (hops) hops[qi] = h;
                if (scored) scored[qi] = sd;
                if (beam_ids) {
                    for (int t = 0; t < L && t < ldb; ++t) {
                        beam_ids[qi * ldb + t] = t < size ? C[t].id : -1;
                        beam_scores[qi * ldb + t] = t < size ? C[t].s : -INFINITY;
                    }
                }
                int nres = 0;
                if (sec && r > 0) {
                    int nc = r < size ? r : size;
                    int rsz = 0;
                    for (int t = 0; t < nc; ++t)
                        cand_insert(R2, &rsz, nc, store_score(sec, qs + qi * (int64_t)sec->dim, C[t].id), C[t].id);
                    for (int t = 0; t < k && t < rsz; ++t) {
                        ids[qi * ldo + t] = R2[t].id;
                        scores[qi * ldo + t] = R2[t].s;
                    }
                    nres = rsz < k ? rsz : k;
                } else {
                    for (int t = 0; t < k && t < size; ++t) {
                        ids[qi * ldo + t] = C[t].id;
                        scores[qi * ldo + t] = C[t].s;
                    }
                    nres = size < k ? size : k;
                }
                for (int t = nres; t < k; ++t) { ids[qi * ldo + t] = -1; scores[qi * ldo + t] = -INFINITY; }
            }
        }
        free(visited); free(C); free(R2);
    }
    return err;
}

/* Exact top-k by <q, x> (metric 0) or by 2 <q, x> - ||x||^2, i.e. by -||q - x||^2 (metric 1),
 * in FP64 over the original vectors (ties -> smaller id). */
int orc_bruteforce(const float *X, int64_t n, const float *Q, int64_t m, int D, int k,
                   int32_t *ids, double *scores, int metric, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    int err = 0;
#pragma omp parallel
    {
        cand_t *C = (cand_t *)malloc(sizeof(cand_t) * (size_t)(k + 1));
        if (!C) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t qi = 0; qi < m; ++qi) {
                int size = 0;
                const float *q = Q + qi * (int64_t)D;
                for (int64_t i = 0; i < n; ++i) {
                    const float *x = X + i * (int64_t)D;
                    double acc = 0.0, nrm = 0.0;
                    for (int j = 0; j < D; ++j) {
                        acc += (double)q[j] * (double)x[j];
                        nrm += (double)x[j] * (double)x[j];
                    }
                    cand_insert(C, &size, k, metric ? 2.0 * acc - nrm : acc, (int32_t)i);
                }
                for (int t = 0; t < k; ++t) {
                    ids[qi * k + t] = t < size ? C[t].id : -1;
                    scores[qi * k + t] = t < size ? C[t].s : -INFINITY;
                }
            }
        }
        free(C);
    }
    return err;
}

/* ------------------------------------------------------------------ */
/* Counter-based SplitMix64 (Steele, Lea, Flood 2014): the k-th output of */
/* the generator seeded with s is mix(s + (k+1) * golden_gamma).          */
/* ------------------------------------------------------------------ */
static uint64_t sm64(uint64_t seed, uint64_t a, uint64_t b)
{
    uint64_t z = seed + 0x9E3779B97F4A7C15ULL * (1ULL + (a << 32) + b);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix(uint64_t seed, uint64_t a, uint64_t b) { return sm64(seed, a, b); }

/* Random initial graph: node v draws ids sm64(seed, v, j) mod n for j = 0,1,..
 * keeping the first min(R, n-1) that are neither v nor already drawn. */
void orc_random_graph(int64_t n, int R, uint64_t seed, int32_t *graph)
{
    int want = (int)((n - 1) < R ? (n - 1) : R);
    for (int64_t v = 0; v < n; ++v) {
        int32_t *row = graph + v * R;
        int cnt = 0;
        for (uint64_t j = 0; cnt < want; ++j) {
            int32_t u = (int32_t)(sm64(seed, (uint64_t)v, j) % (uint64_t)n);
            if (u == v) continue;
            int dup = 0;
            for (int t = 0; t < cnt; ++t) if (row[t] == u) { dup = 1; break; }
            if (dup) continue;
            row[cnt++] = u;
        }
        for (int t = cnt; t < R; ++t) row[t] = -1;
    }
}

/* Fisher-Yates permutation with draws sm64(seed + 1, i, 0) mod (i + 1). */
void orc_permutation(int64_t n, uint64_t seed, int32_t *perm)
{
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i >= 1; --i) {
        int64_t j = (int64_t)(sm64(seed + 1, (uint64_t)i, 0) % (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* ------------------------------------------------------------------ */
/* RobustPrune (App. A "Pruning"; inner-product forms of the DiskANN rule): */
/* sort the pool by s(p, .) desc (id asc); repeatedly keep the best      */
/* remaining p* and drop every remaining p' with                        */
/*   alpha * s(p*,p') >= s(p,p') + shift                                 */
/* shift = 0 (alpha scales the similarity) or alpha - 1 (the L2 rule     */
/* alpha d(p*,p') <= d(p,p') with d = 2 - 2 s, i.e. unit-norm vectors).  */
/* The pool must exclude p and hold distinct ids.  Returns |N| <= R.     */
/* ------------------------------------------------------------------ */
static int robust_prune(const orc_bstore *bs, int32_t p, const int32_t *pool, int np,
                        float alpha, float shift, int R, int32_t *out)
{
    cand_t *V = (cand_t *)malloc(sizeof(cand_t) * (size_t)(np + 1));
    int nv = 0;
    for (int t = 0; t < np; ++t) cand_insert(V, &nv, np, (double)bscore(bs, p, pool[t]), pool[t]);
    int nout = 0;
    for (int i = 0; i < nv && nout < R; ++i) {
        if (V[i].expanded) continue;            /* 'expanded' marks removed */
        out[nout++] = V[i].id;
        for (int j = i + 1; j < nv; ++j) {
            if (V[j].expanded) continue;
            float sps = bscore(bs, V[i].id, V[j].id);
            float lhs = alpha * sps;
            float rhs = (float)V[j].s + shift;
            if (lhs >= rhs) V[j].expanded = 1;
        }
    }
    free(V);
    return nout;
}

int orc_robust_prune(const uint8_t *codes, const float *delta, const float *lower,
                     const float *G, const float *H, const float *N, float mu2, int dim,
                     int32_t p, const int32_t *pool, int np, float alpha, float shift, int R, int32_t *out)
{
    orc_bstore bs = {dim, codes, delta, lower, (float *)G, (float *)H, N, mu2};
    return robust_prune(&bs, p, pool, np, alpha, shift, R, out);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* inner product: entry = argmax_i <mean, y_i> over decoded primaries, i.e. argmax G_i;
 * L2 (N != NULL): the primary nearest the mean, argmin ||y_i - mean||^2 =
 * argmax 2 G_i - N_i (FP32); ties -> smaller id. */
int32_t orc_entry_point(const float *G, const float *N, int64_t n)
{
    int32_t best = 0;
    float kb = N ? 2.0f * G[0] - N[0] : G[0];
    for (int64_t i = 1; i < n; ++i) {
        const float ki = N ? 2.0f * G[i] - N[i] : G[i];
        if (ki > kb) { best = (int32_t)i; kb = ki; }
    }
    return best;
}

/*
 * Batch-synchronous Vamana on primary vectors (App. A: search + prune per
 * node; App. D: R, L, alpha).  Pass t uses alpha_t = 1 for t < passes-1 and
 * alpha for the last pass; rule 0 prunes with shift 0, rule 1 with shift alpha_t - 1.  Each batch of `batch` nodes (in permutation order)
 *   1. searches, from the entry, the graph as it was at the start of the batch
 *      (query = the node's own primary, beam L_build, no rerank);
 *   2. prunes pool = beam ∪ old out-neighbours (minus the node) to <= R;
 *   3. replaces the batch nodes' out-lists;
 *   4. applies reverse edges by target u ascending: the sources p (ascending)
 *      not already listed are appended; if u then has more than R
 *      out-neighbours, its list is pruned with its own list as the pool.
 * batch = 1 is the sequential algorithm.  graph: n x R, -1 padded, in/out.
 */
int orc_vamana_build(const uint8_t *codes, const float *delta, const float *lower,
                     const float *G, const float *H, const float *N, float mu2, int dim, int64_t n,
                     int R, int L_build, float alpha, int passes, int batch, uint64_t seed, int rule,
                     int32_t *graph, int32_t *entry_out, int nthreads)
{
    orc_bstore bs = {dim, codes, delta, lower, (float *)G, (float *)H, N, mu2};
    if (batch < 1 || R < 1 || L_build < 1 || passes < 1) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    orc_random_graph(n, R, seed, graph);
    int32_t entry = orc_entry_point(G, N, n);
    *entry_out = entry;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *snap = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * R);
    int32_t *newl = (int32_t *)malloc(sizeof(int32_t) * (size_t)batch * R);
    int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)batch * R);
    if (!perm || !snap || !newl || !pairs) return -2;
    orc_permutation(n, seed, perm);

    for (int pass = 0; pass < passes; ++pass) {
        float a = (pass < passes - 1) ? 1.0f : alpha;
        float shift = rule ? a - 1.0f : 0.0f;
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            int nb = (int)((n - b0) < batch ? (n - b0) : batch);
            memcpy(snap, graph, sizeof(int32_t) * (size_t)n * R);
            int err = 0;
#pragma omp parallel
            {
                uint32_t *visited = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
                cand_t *C = (cand_t *)malloc(sizeof(cand_t) * (size_t)(L_build + 1));
                int32_t *pool = (int32_t *)malloc(sizeof(int32_t) * (size_t)(L_build + R));
                uint32_t stamp = 0;
                if (!visited || !C || !pool) {
#pragma omp atomic write
                    err = -2;
                } else {
#pragma omp for schedule(dynamic, 1)
                    for (int t = 0; t < nb; ++t) {
                        int32_t p = perm[b0 + t];
                        stamp++;
                        scorer_t sc = {NULL, NULL, &bs, p};
                        int size = beam_search(&sc, snap, R, n, entry, L_build, 0, 1, visited, stamp, C, NULL, NULL);
                        int np = 0;
                        for (int s = 0; s < size; ++s) if (C[s].id != p) pool[np++] = C[s].id;
                        for (int s = 0; s < R; ++s) {
                            int32_t u = snap[(int64_t)p * R + s];
                            if (u < 0 || u == p) continue;
                            int dup = 0;
                            for (int w = 0; w < np; ++w) if (pool[w] == u) { dup = 1; break; }
                            if (!dup) pool[np++] = u;
                        }
                        int32_t *out = newl + (int64_t)t * R;
                        int no = robust_prune(&bs, p, pool, np, a, shift, R, out);
                        for (int s = no; s < R; ++s) out[s] = -1;
                    }
                }
                free(visited); free(C); free(pool);
            }
            if (err) return err;
            /* 3. replace the batch's out-lists */
            for (int t = 0; t < nb; ++t)
                memcpy(graph + (int64_t)perm[b0 + t] * R, newl + (int64_t)t * R, sizeof(int32_t) * R);
            /* 4. reverse edges, by (target, source) ascending */
            int np2 = 0;
            for (int t = 0; t < nb; ++t) {
                int32_t p = perm[b0 + t];
                for (int s = 0; s < R; ++s) {
                    int32_t u = graph[(int64_t)p * R + s];
                    if (u < 0) continue;
                    pairs[2 * np2] = u; pairs[2 * np2 + 1] = p; np2++;
                }
            }
            /* sort pairs by (u, p): both are non-negative, so packing u in the
             * high and p in the low 32 bits orders the int64 keys by (u, p) */
            int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np2 + 1));
            for (int t = 0; t < np2; ++t) keys[t] = ((int64_t)pairs[2 * t] << 32) | (uint32_t)pairs[2 * t + 1];
            qsort(keys, (size_t)np2, sizeof(int64_t), cmp_i64);
            int t0 = 0;
            int32_t *lst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R + batch + 1));
            int32_t *pr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R + batch + 1));
            while (t0 < np2) {
                int32_t u = (int32_t)(keys[t0] >> 32);
                int t1 = t0;
                while (t1 < np2 && (int32_t)(keys[t1] >> 32) == u) t1++;
                int nl = 0;
                for (int s = 0; s < R; ++s) {
                    int32_t w = graph[(int64_t)u * R + s];
                    if (w >= 0) lst[nl++] = w;
                }
                for (int t = t0; t < t1; ++t) {
                    int32_t p = (int32_t)(keys[t] & 0xffffffff);
                    if (p == u) continue;
                    int dup = 0;
                    for (int w = 0; w < nl; ++w) if (lst[w] == p) { dup = 1; break; }
                    if (!dup) lst[nl++] = p;
                }
                if (nl > R) {
                    int no = robust_prune(&bs, u, lst, nl, a, shift, R, pr);
                    for (int s = 0; s < R; ++s) graph[(int64_t)u * R + s] = s < no ? pr[s] : -1;
                } else {
                    for (int s = 0; s < R; ++s) graph[(int64_t)u * R + s] = s < nl ? lst[s] : -1;
                }
                t0 = t1;
            }
            free(lst); free(pr); free(keys);
        }
    }
    free(perm); free(snap); free(newl); free(pairs);
    return 0;
}


/*
 * CPU oracle for layered min-sum decoding of quasi-cyclic LDPC codes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header, table or
 * helper with the CUDA decoder; both sides only receive the same seeded inputs.
 *
 * It runs the method exactly as written in the paper, scalar, one codeword at a time:
 *
 *   Sec. II   code model: base graph rows r, columns c, circulant shift s; check row i of
 *             block (r, c) connects variable c*Z + ((i + s) mod Z); the first `punct`
 *             columns are punctured (their channel LLR is 0).
 *   Sec. III  check node (min-sum with correction beta):
 *                 L_c->v^i = beta * min_{j != i} |L_v->c^j| * prod_{j != i} sgn(L_v->c^j)
 *             posterior       L_v = L_b + sum_k L_c->v^k
 *             next message    L_v->c^i = L_v^i - L_c->v^i
 *             layered schedule: base rows one at a time in natural order, each row's
 *             update visible to the next; stop at a valid codeword or the iteration cap.
 *   Sec. IV   the per-row quantities m1 (min), m2 (min over i != argmin), the sign product
 *             of the incoming messages, and the row parity of the posteriors' hard
 *             decisions (used for the stopping test).
 *
 * Readings where the paper is silent (listed again in the design notes):
 *   - sgn(0) = +1; hard decision bit = (L_v < 0).
 *   - argmin ties go to the lowest edge index (edges of a row in increasing column order);
 *     forward messages do not depend on it because m2 = m1 on a tie.
 *   - corrections: normalised  m' = alpha * m          (fp32 / fp16)
 *                  offset      m' = max(m - offset, 0) (int8 units, or LLR units in fp)
 *                  learned     m' = beta[t][r] * max(m - gamma[t][r], 0)   (fp32)
 *   - int8: L_v, v->c and c->v saturate to [-127, 127] (-128 never used).
 *   - fp16: every stored message and posterior is rounded to binary16 (round to nearest
 *     even) after each operation; the rounding is written from the IEEE 754 definition.
 *     The correction parameters (alpha, offset, beta, gamma) are rounded to binary16 once.
 *   - stopping: after every full iteration the syndrome of the hard decisions over the
 *     used rows is computed; all zero ends decoding (no test before iteration 1).  A
 *     stopped codeword's posteriors are frozen; iterations = number executed.
 *   - hard-bit output: the first K = K_b * Z bits, punctured ones included.
 *
 * Everything here is plain C99, -O2, no vectorisation pragmas; fp32 code is compiled with
 * -ffp-contract=off so every operation rounds once, as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_LLR_INT8 = 0, OR_LLR_FP16 = 1, OR_LLR_FP32 = 2 };
enum { OR_NORMALISED = 0, OR_OFFSET = 1, OR_LEARNED = 2 };
enum { OR_OK = 0, OR_BAD_ARG = 1, OR_NO_MEM = 2 };

typedef struct {
    int Z;
    int n_rows;    /* base rows used */
    int n_cols;    /* base columns used = K_b + n_rows */
    int K_b;
    int E;         /* edges (non-zero circulants) in the used rows */
    int *row_ptr;  /* n_rows + 1 */
    int *col;      /* E */
    int *shift;    /* E, already reduced mod Z */
} og_graph;

static void graph_free(og_graph *g)
{
    free(g->row_ptr);
    free(g->col);
    free(g->shift);
}

/* Edge lists of the first n_rows base rows, each row's edges in increasing column order. */
static int graph_build(const int16_t *base, int M_bg, int N_bg, int K_b, int Z, int n_rows,
                       og_graph *g)
{
    memset(g, 0, sizeof(*g));
    if (!base || Z < 1 || n_rows < 1 || n_rows > M_bg || K_b < 1 || K_b + n_rows > N_bg)
        return OR_BAD_ARG;
    g->Z = Z;
    g->n_rows = n_rows;
    g->K_b = K_b;
    g->n_cols = K_b + n_rows;
    int E = 0;
    for (int r = 0; r < n_rows; ++r)
        for (int c = 0; c < N_bg; ++c)
            if (base[r * N_bg + c] >= 0) {
                if (c >= g->n_cols)
                    return OR_BAD_ARG;
                ++E;
            }
    g->E = E;
    g->row_ptr = (int *)malloc(sizeof(int) * (n_rows + 1));
    g->col = (int *)malloc(sizeof(int) * (E ? E : 1));
    g->shift = (int *)malloc(sizeof(int) * (E ? E : 1));
    if (!g->row_ptr || !g->col || !g->shift) {
        graph_free(g);
        return OR_NO_MEM;
    }
    int e = 0;
    for (int r = 0; r < n_rows; ++r) {
        g->row_ptr[r] = e;
        for (int c = 0; c < N_bg; ++c) {
            int v = base[r * N_bg + c];
            if (v >= 0) {
                g->col[e] = c;
                g->shift[e] = v % Z;
                ++e;
            }
        }
    }
    g->row_ptr[n_rows] = e;
    for (int r = 0; r < n_rows; ++r)
        if (g->row_ptr[r + 1] - g->row_ptr[r] < 2) {   /* min over the other edges must exist */
            graph_free(g);
            return OR_BAD_ARG;
        }
    return OR_OK;
}

/* variable node touched by check row i of edge e */
static int var_of(const og_graph *g, int e, int i)
{
    return g->col[e] * g->Z + (i + g->shift[e]) % g->Z;
}

/* ---------------------------------------------------------------- arithmetic helpers */

static int sat8(int x)
{
    return x > 127 ? 127 : (x < -127 ? -127 : x);
}

/* Round a real value to the nearest binary16 value, ties to even (IEEE 754-2008, 4.3.1).
 * Binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits; normal numbers have
 * quantum 2^(e-10) in binade [2^e, 2^(e+1)), e >= -14; below 2^-14 the quantum is 2^-24.
 * The largest finite value is 65504; anything that rounds beyond it becomes infinity. */
static float round_half(double x)
{
    if (x != x)
        return (float)x;
    double a = fabs(x);
    if (a == 0.0)
        return (float)x;
    int e;
    frexp(a, &e);           /* a = f * 2^e, f in [0.5, 1) -> a in [2^(e-1), 2^e) */
    int binade = e - 1;     /* a in [2^binade, 2^(binade+1)) */
    if (binade < -14)
        binade = -14;       /* subnormal range shares the quantum of the lowest binade */
    double q = ldexp(1.0, binade - 10);
    double r = nearbyint(a / q) * q;   /* default rounding mode: to nearest, ties to even */
    if (r > 65504.0)
        r = INFINITY;
    return (float)(x < 0 ? -r : r);
}

/* binary16 bit pattern <-> value (exact; used only for input/output marshalling) */
static float half_bits_to_float(uint16_t h)
{
    int s = h >> 15, ex = (h >> 10) & 31, fr = h & 1023;
    double v;
    if (ex == 0)
        v = ldexp((double)fr, -24);
    else if (ex == 31)
        v = fr ? NAN : INFINITY;
    else
        v = ldexp((double)(fr + 1024), ex - 25);
    return (float)(s ? -v : v);
}

static uint16_t float_to_half_bits(float f)
{
    /* f is already a binary16 value (or +-inf); encode it exactly */
    uint16_t s = signbit(f) ? 0x8000 : 0;
    double a = fabs((double)f);
    if (isinf(f))
        return s | 0x7C00;
    if (a != a)
        return 0x7E00;
    if (a == 0.0)
        return s;
    int e;
    double fr = frexp(a, &e);       /* a = fr * 2^e */
    int ex = e - 1 + 15;            /* biased exponent of [2^(e-1), 2^e) */
    if (ex <= 0)                    /* subnormal: a = m * 2^-24 */
        return s | (uint16_t)(a / ldexp(1.0, -24));
    int m = (int)(fr * 2048.0) - 1024;
    return s | (uint16_t)(ex << 10) | (uint16_t)m;
}

/* --------------------------------------------------------- check-node update (Sec. III/IV)
 *
 * Input: the d variable-to-check messages of one check row (already in the working
 * precision).  Output: the d check-to-variable messages, using the four per-row
 * quantities of Sec. IV: m1 = min |v|, idx = argmin (lowest index on ties),
 * m2 = min over i != idx, S = parity of the negative messages.  For edge i the magnitude
 * is m2 if i == idx else m1 (min over j != i), the sign is S xor sgn(v_i)
 * (product over j != i), and the correction is applied to the magnitude.
 */
typedef struct {
    int mode;        /* OR_NORMALISED / OR_OFFSET / OR_LEARNED */
    float alpha;     /* normalised */
    float offset;    /* offset (fp: LLR units) */
    int offset_q;    /* offset (int8 units) */
    float beta, gamma;   /* learned, for the current (iteration, row) */
} cn_corr;

static float corr_f32(const cn_corr *c, float m)
{
    switch (c->mode) {
    case OR_NORMALISED:
        return c->alpha * m;
    case OR_OFFSET: {
        float t = m - c->offset;
        return t > 0.0f ? t : 0.0f;
    }
    default: {
        float t = m - c->gamma;
        t = t > 0.0f ? t : 0.0f;
        return c->beta * t;
    }
    }
}

static int corr_i8(const cn_corr *c, int m)
{
    int t = m - c->offset_q;
    return t > 0 ? t : 0;
}

/* binary16 path: the correction parameters are themselves binary16 values (each rounded
 * once from its fp32 input), so every step of the check rule is one binary16 operation. */
static float corr_f16(const cn_corr *c, float m)
{
    switch (c->mode) {
    case OR_NORMALISED:
        return round_half((double)round_half(c->alpha) * (double)m);
    case OR_OFFSET: {
        float t = round_half((double)m - (double)round_half(c->offset));
        return t > 0.0f ? t : 0.0f;
    }
    default: {
        float t = round_half((double)m - (double)round_half(c->gamma));
        t = t > 0.0f ? t : 0.0f;
        return round_half((double)round_half(c->beta) * (double)t);
    }
    }
}

void oracle_check_node_f32(const float *v, int d, int mode, float alpha, float offset,
                           float beta, float gamma, float *out)
{
    cn_corr c = {mode, alpha, offset, 0, beta, gamma};
    float m1 = INFINITY, m2 = INFINITY;
    int idx = -1, S = 0;
    for (int k = 0; k < d; ++k) {
        float a = fabsf(v[k]);
        if (a < m1) {
            m2 = m1;
            m1 = a;
            idx = k;
        } else if (a < m2) {
            m2 = a;
        }
        S ^= (v[k] < 0.0f);
    }
    float m1c = corr_f32(&c, m1), m2c = corr_f32(&c, m2);
    for (int k = 0; k < d; ++k) {
        float mag = (k == idx) ? m2c : m1c;
        int neg = S ^ (v[k] < 0.0f);
        out[k] = neg ? -mag : mag;
    }
}

void oracle_check_node_i8(const int8_t *v, int d, int offset_q, int8_t *out)
{
    cn_corr c = {OR_OFFSET, 0.f, 0.f, offset_q, 0.f, 0.f};
    int m1 = 1 << 20, m2 = 1 << 20, idx = -1, S = 0;
    for (int k = 0; k < d; ++k) {
        int a = v[k] < 0 ? -v[k] : v[k];
        if (a < m1) {
            m2 = m1;
            m1 = a;
            idx = k;
        } else if (a < m2) {
            m2 = a;
        }
        S ^= (v[k] < 0);
    }
    int m1c = corr_i8(&c, m1), m2c = corr_i8(&c, m2);
    for (int k = 0; k < d; ++k) {
        int mag = (k == idx) ? m2c : m1c;
        int neg = S ^ (v[k] < 0);
        out[k] = (int8_t)(neg ? -mag : mag);
    }
}

/* --------------------------------------------------------------- syndrome (Sec. III/IV)
 * Parity of the hard decisions (bit = L_v < 0) of every used check row; returns the number
 * of unsatisfied check rows. */
static int syndrome_weight_f(const og_graph *g, const float *Lv)
{
    int bad = 0;
    for (int r = 0; r < g->n_rows; ++r)
        for (int i = 0; i < g->Z; ++i) {
            int p = 0;
            for (int e = g->row_ptr[r]; e < g->row_ptr[r + 1]; ++e)
                p ^= (Lv[var_of(g, e, i)] < 0.0f);
            bad += p;
        }
    return bad;
}

static int syndrome_weight_i8(const og_graph *g, const int8_t *Lv)
{
    int bad = 0;
    for (int r = 0; r < g->n_rows; ++r)
        for (int i = 0; i < g->Z; ++i) {
            int p = 0;
            for (int e = g->row_ptr[r]; e < g->row_ptr[r + 1]; ++e)
                p ^= (Lv[var_of(g, e, i)] < 0);
            bad += p;
        }
    return bad;
}

/* Syndrome weight of hard-decision words (uint8 bits [n_cols*Z]) — used by the tests to
 * check codewords and decoder outputs. */
int oracle_syndrome_bits(const int16_t *base, int M_bg, int N_bg, int K_b, int Z, int n_rows,
                         const uint8_t *bits)
{
    og_graph g;
    if (graph_build(base, M_bg, N_bg, K_b, Z, n_rows, &g) != OR_OK)
        return -1;
    int bad = 0;
    for (int r = 0; r < g.n_rows; ++r)
        for (int i = 0; i < Z; ++i) {
            int p = 0;
            for (int e = g.row_ptr[r]; e < g.row_ptr[r + 1]; ++e)
                p ^= bits[var_of(&g, e, i)] & 1;
            bad += p;
        }
    graph_free(&g);
    return bad;
}

/* -------------------------------------------------------------------- decode: common */

typedef struct {
    int punct;           /* punctured leading columns */
    int n_tx;            /* channel LLRs per codeword */
    int max_iter;
    int early_stop;
    cn_corr corr;
    const float *learned;   /* [max_iter][n_rows][2] (beta, gamma) or NULL */
} dec_cfg;

static int dec_max_degree(const og_graph *g)
{
    int d = 0;
    for (int r = 0; r < g->n_rows; ++r)
        if (g->row_ptr[r + 1] - g->row_ptr[r] > d)
            d = g->row_ptr[r + 1] - g->row_ptr[r];
    return d;
}

/* ------------------------------------------------------------------ decode: fp32 path */
static void decode_one_f32(const og_graph *g, const dec_cfg *cfg, const float *llr, float *Lv,
                           float *c2v, float *v, uint8_t *bits, int32_t *iters)
{
    const int Z = g->Z, N = g->n_cols * Z;
    for (int j = 0; j < N; ++j)
        Lv[j] = 0.0f;
    for (int j = 0; j < cfg->n_tx; ++j)
        Lv[cfg->punct * Z + j] = llr[j];
    for (int k = 0; k < g->E * Z; ++k)
        c2v[k] = 0.0f;
    int done = cfg->max_iter;
    for (int t = 1; t <= cfg->max_iter; ++t) {
        for (int r = 0; r < g->n_rows; ++r) {
            cn_corr c = cfg->corr;
            if (c.mode == OR_LEARNED) {
                c.beta = cfg->learned[((t - 1) * g->n_rows + r) * 2 + 0];
                c.gamma = cfg->learned[((t - 1) * g->n_rows + r) * 2 + 1];
            }
            const int e0 = g->row_ptr[r], d = g->row_ptr[r + 1] - e0;
            for (int i = 0; i < Z; ++i) {
                /* variable-to-check messages (Sec. III, L_v->c = L_v - L_c->v) */
                for (int k = 0; k < d; ++k)
                    v[k] = Lv[var_of(g, e0 + k, i)] - c2v[(e0 + k) * Z + i];
                /* check node */
                float m1 = INFINITY, m2 = INFINITY;
                int idx = -1, S = 0;
                for (int k = 0; k < d; ++k) {
                    float a = fabsf(v[k]);
                    if (a < m1) {
                        m2 = m1;
                        m1 = a;
                        idx = k;
                    } else if (a < m2) {
                        m2 = a;
                    }
                    S ^= (v[k] < 0.0f);
                }
                float m1c = corr_f32(&c, m1), m2c = corr_f32(&c, m2);
                /* new check-to-variable messages and posterior write-back */
                for (int k = 0; k < d; ++k) {
                    float mag = (k == idx) ? m2c : m1c;
                    float cv = (S ^ (v[k] < 0.0f)) ? -mag : mag;
                    c2v[(e0 + k) * Z + i] = cv;
                    Lv[var_of(g, e0 + k, i)] = v[k] + cv;
                }
            }
        }
        if (cfg->early_stop && syndrome_weight_f(g, Lv) == 0) {
            done = t;
            break;
        }
    }
    for (int j = 0; j < g->K_b * Z; ++j)
        bits[j] = (Lv[j] < 0.0f);
    *iters = done;
}

/* ------------------------------------------------------------------ decode: fp16 path */
static void decode_one_f16(const og_graph *g, const dec_cfg *cfg, const float *llr, float *Lv,
                           float *c2v, float *v, uint8_t *bits, int32_t *iters)
{
    const int Z = g->Z, N = g->n_cols * Z;
    for (int j = 0; j < N; ++j)
        Lv[j] = 0.0f;
    for (int j = 0; j < cfg->n_tx; ++j)
        Lv[cfg->punct * Z + j] = llr[j];     /* already binary16 values */
    for (int k = 0; k < g->E * Z; ++k)
        c2v[k] = 0.0f;
    int done = cfg->max_iter;
    for (int t = 1; t <= cfg->max_iter; ++t) {
        for (int r = 0; r < g->n_rows; ++r) {
            cn_corr c = cfg->corr;
            if (c.mode == OR_LEARNED) {
                c.beta = cfg->learned[((t - 1) * g->n_rows + r) * 2 + 0];
                c.gamma = cfg->learned[((t - 1) * g->n_rows + r) * 2 + 1];
            }
            const int e0 = g->row_ptr[r], d = g->row_ptr[r + 1] - e0;
            for (int i = 0; i < Z; ++i) {
                for (int k = 0; k < d; ++k)
                    v[k] = round_half((double)Lv[var_of(g, e0 + k, i)] -
                                      (double)c2v[(e0 + k) * Z + i]);
                float m1 = INFINITY, m2 = INFINITY;
                int idx = -1, S = 0;
                for (int k = 0; k < d; ++k) {
                    float a = fabsf(v[k]);
                    if (a < m1) {
                        m2 = m1;
                        m1 = a;
                        idx = k;
                    } else if (a < m2) {
                        m2 = a;
                    }
                    S ^= (v[k] < 0.0f);
                }
                float m1c = corr_f16(&c, m1), m2c = corr_f16(&c, m2);
                for (int k = 0; k < d; ++k) {
                    float mag = (k == idx) ? m2c : m1c;
                    float cv = (S ^ (v[k] < 0.0f)) ? -mag : mag;
                    c2v[(e0 + k) * Z + i] = cv;
                    Lv[var_of(g, e0 + k, i)] = round_half((double)v[k] + (double)cv);
                }
            }
        }
        if (cfg->early_stop && syndrome_weight_f(g, Lv) == 0) {
            done = t;
            break;
        }
    }
    for (int j = 0; j < g->K_b * Z; ++j)
        bits[j] = (Lv[j] < 0.0f);
    *iters = done;
}

/* ------------------------------------------------------------------ decode: int8 path */
static void decode_one_i8(const og_graph *g, const dec_cfg *cfg, const int8_t *llr, int8_t *Lv,
                          int8_t *c2v, int *v, uint8_t *bits, int32_t *iters)
{
    const int Z = g->Z, N = g->n_cols * Z;
    memset(Lv, 0, (size_t)N);
    for (int j = 0; j < cfg->n_tx; ++j)
        Lv[cfg->punct * Z + j] = (int8_t)sat8(llr[j]);
    memset(c2v, 0, (size_t)g->E * Z);
    int done = cfg->max_iter;
    for (int t = 1; t <= cfg->max_iter; ++t) {
        for (int r = 0; r < g->n_rows; ++r) {
            const int e0 = g->row_ptr[r], d = g->row_ptr[r + 1] - e0;
            for (int i = 0; i < Z; ++i) {
                for (int k = 0; k < d; ++k)
                    v[k] = sat8(Lv[var_of(g, e0 + k, i)] - c2v[(e0 + k) * Z + i]);
                int m1 = 1 << 20, m2 = 1 << 20, idx = -1, S = 0;
                for (int k = 0; k < d; ++k) {
                    int a = v[k] < 0 ? -v[k] : v[k];
                    if (a < m1) {
                        m2 = m1;
                        m1 = a;
                        idx = k;
                    } else if (a < m2) {
                        m2 = a;
                    }
                    S ^= (v[k] < 0);
                }
                int m1c = corr_i8(&cfg->corr, m1), m2c = corr_i8(&cfg->corr, m2);
                for (int k = 0; k < d; ++k) {
                    int mag = (k == idx) ? m2c : m1c;
                    int cv = (S ^ (v[k] < 0)) ? -mag : mag;
                    c2v[(e0 + k) * Z + i] = (int8_t)cv;
                    Lv[var_of(g, e0 + k, i)] = (int8_t)sat8(v[k] + cv);
                }
            }
        }
        if (cfg->early_stop && syndrome_weight_i8(g, Lv) == 0) {
            done = t;
            break;
        }
    }
    for (int j = 0; j < g->K_b * Z; ++j)
        bits[j] = (Lv[j] < 0);
    *iters = done;
}

/* ------------------------------------------------------------------ public entry point
 *
 * llr:   [batch][n_tx] of int8 / binary16 bits (uint16) / float32 per llr_type
 * bits:  [batch][K_b*Z] uint8, one hard decision per byte (0/1)
 * iters: [batch] int32
 * post:  optional [batch][(K_b+n_rows)*Z] posteriors in the llr type (uint16 for fp16)
 * c2v:   optional [batch][E*Z] check-to-variable messages, edge-major (edge*Z + row)
 * cw_begin/cw_end: decode only codewords [cw_begin, cw_end) (lets callers thread over the
 *   batch); outputs are indexed by the absolute codeword number.
 */
int oracle_decode_layered(const int16_t *base, int M_bg, int N_bg, int K_b, int Z, int n_rows,
                          int punct, int n_tx, int llr_type, int algo, float alpha,
                          float offset, int offset_q, const float *learned, int max_iter,
                          int early_stop, const void *llr, int cw_begin, int cw_end,
                          uint8_t *bits, int32_t *iters, void *post, void *c2v_out)
{
    og_graph g;
    int st = graph_build(base, M_bg, N_bg, K_b, Z, n_rows, &g);
    if (st != OR_OK)
        return st;
    const int N = g.n_cols * Z, K = K_b * Z, EZ = g.E * Z;
    if (punct < 0 || n_tx < 0 || punct * Z + n_tx > N || max_iter < 1 || cw_begin < 0 ||
        cw_end < cw_begin || (algo == OR_LEARNED && !learned) ||
        (llr_type == OR_LLR_INT8 && algo != OR_OFFSET) || llr_type < 0 || llr_type > 2) {
        graph_free(&g);
        return OR_BAD_ARG;
    }
    dec_cfg cfg;
    cfg.punct = punct;
    cfg.n_tx = n_tx;
    cfg.max_iter = max_iter;
    cfg.early_stop = early_stop;
    cfg.corr.mode = algo;
    cfg.corr.alpha = alpha;
    cfg.corr.offset = offset;
    cfg.corr.offset_q = offset_q;
    cfg.corr.beta = 0.f;
    cfg.corr.gamma = 0.f;
    cfg.learned = learned;
    const int dmax = dec_max_degree(&g);
    float *Lf = NULL, *Cf = NULL, *vf = NULL, *lb = NULL;
    int8_t *Li = NULL, *Ci = NULL;
    int *vi = NULL;
    int ok = 1;
    if (llr_type == OR_LLR_INT8) {
        Li = (int8_t *)malloc((size_t)N);
        Ci = (int8_t *)malloc((size_t)EZ + 1);
        vi = (int *)malloc(sizeof(int) * (dmax + 1));
        ok = Li && Ci && vi;
    } else {
        Lf = (float *)malloc(sizeof(float) * N);
        Cf = (float *)malloc(sizeof(float) * (EZ + 1));
        vf = (float *)malloc(sizeof(float) * (dmax + 1));
        lb = (float *)malloc(sizeof(float) * (n_tx + 1));
        ok = Lf && Cf && vf && lb;
    }
    if (!ok) {
        free(Li); free(Ci); free(vi); free(Lf); free(Cf); free(vf); free(lb);
        graph_free(&g);
        return OR_NO_MEM;
    }
    for (int b = cw_begin; b < cw_end; ++b) {
        uint8_t *bb = bits + (size_t)b * K;
        int32_t *it = iters + b;
        if (llr_type == OR_LLR_INT8) {
            decode_one_i8(&g, &cfg, (const int8_t *)llr + (size_t)b * n_tx, Li, Ci, vi, bb, it);
            if (post)
                memcpy((int8_t *)post + (size_t)b * N, Li, (size_t)N);
            if (c2v_out)
                memcpy((int8_t *)c2v_out + (size_t)b * EZ, Ci, (size_t)EZ);
        } else if (llr_type == OR_LLR_FP32) {
            decode_one_f32(&g, &cfg, (const float *)llr + (size_t)b * n_tx, Lf, Cf, vf, bb, it);
            if (post)
                memcpy((float *)post + (size_t)b * N, Lf, sizeof(float) * N);
            if (c2v_out)
                memcpy((float *)c2v_out + (size_t)b * EZ, Cf, sizeof(float) * EZ);
        } else {
            const uint16_t *h = (const uint16_t *)llr + (size_t)b * n_tx;
            for (int j = 0; j < n_tx; ++j)
                lb[j] = half_bits_to_float(h[j]);
            decode_one_f16(&g, &cfg, lb, Lf, Cf, vf, bb, it);
            if (post)
                for (int j = 0; j < N; ++j)
                    ((uint16_t *)post)[(size_t)b * N + j] = float_to_half_bits(Lf[j]);
            if (c2v_out)
                for (int k = 0; k < EZ; ++k)
                    ((uint16_t *)c2v_out)[(size_t)b * EZ + k] = float_to_half_bits(Cf[k]);
        }
    }
    free(Li); free(Ci); free(vi); free(Lf); free(Cf); free(vf); free(lb);
    graph_free(&g);
    return OR_OK;
}

/* ------------------------------------------------------- flooding schedule (Sec. III)
 * All check rows of all used base rows are updated from the same posteriors, then every
 * posterior is recomputed as L_b + sum of the new check-to-variable messages.  fp32,
 * min-sum with the same corrections as the layered decoder, or exact sum-product
 * (algo = 3: L_c->v^i = 2 atanh(prod_{j != i} tanh(L_v->c^j / 2)), computed in double).
 */
enum { OR_SUM_PRODUCT = 3 };

int oracle_decode_flooding(const int16_t *base, int M_bg, int N_bg, int K_b, int Z, int n_rows,
                           int punct, int n_tx, int algo, float alpha, float offset,
                           int max_iter, int early_stop, const float *llr, int cw_begin,
                           int cw_end, uint8_t *bits, int32_t *iters, float *post)
{
    og_graph g;
    int st = graph_build(base, M_bg, N_bg, K_b, Z, n_rows, &g);
    if (st != OR_OK)
        return st;
    const int N = g.n_cols * Z, K = K_b * Z, EZ = g.E * Z;
    if (punct < 0 || n_tx < 0 || punct * Z + n_tx > N || max_iter < 1 || algo == OR_LEARNED) {
        graph_free(&g);
        return OR_BAD_ARG;
    }
    cn_corr corr = {algo, alpha, offset, 0, 0.f, 0.f};
    const int dmax = dec_max_degree(&g);
    float *Lb = (float *)malloc(sizeof(float) * N);
    float *Lv = (float *)malloc(sizeof(float) * N);
    float *c2v = (float *)malloc(sizeof(float) * (EZ + 1));
    float *v = (float *)malloc(sizeof(float) * (dmax + 1));
    double *tv = (double *)malloc(sizeof(double) * (dmax + 1));
    if (!Lb || !Lv || !c2v || !v || !tv) {
        free(Lb); free(Lv); free(c2v); free(v); free(tv);
        graph_free(&g);
        return OR_NO_MEM;
    }
    for (int b = cw_begin; b < cw_end; ++b) {
        for (int j = 0; j < N; ++j)
            Lb[j] = 0.0f;
        for (int j = 0; j < n_tx; ++j)
            Lb[punct * Z + j] = llr[(size_t)b * n_tx + j];
        for (int j = 0; j < N; ++j)
            Lv[j] = Lb[j];
        for (int k = 0; k < EZ; ++k)
            c2v[k] = 0.0f;
        int done = max_iter;
        for (int t = 1; t <= max_iter; ++t) {
            /* all check nodes from the posteriors of the previous iteration */
            for (int r = 0; r < g.n_rows; ++r) {
                const int e0 = g.row_ptr[r], d = g.row_ptr[r + 1] - e0;
                for (int i = 0; i < Z; ++i) {
                    for (int k = 0; k < d; ++k)
                        v[k] = Lv[var_of(&g, e0 + k, i)] - c2v[(e0 + k) * Z + i];
                    if (algo == OR_SUM_PRODUCT) {
                        for (int k = 0; k < d; ++k)
                            tv[k] = tanh(0.5 * (double)v[k]);
                        for (int k = 0; k < d; ++k) {
                            double p = 1.0;
                            for (int j = 0; j < d; ++j)
                                if (j != k)
                                    p *= tv[j];
                            if (p > 1.0 - 1e-15)
                                p = 1.0 - 1e-15;
                            if (p < -1.0 + 1e-15)
                                p = -1.0 + 1e-15;
                            c2v[(e0 + k) * Z + i] = (float)(2.0 * atanh(p));
                        }
                    } else {
                        float m1 = INFINITY, m2 = INFINITY;
                        int idx = -1, S = 0;
                        for (int k = 0; k < d; ++k) {
                            float a = fabsf(v[k]);
                            if (a < m1) {
                                m2 = m1;
                                m1 = a;
                                idx = k;
                            } else if (a < m2) {
                                m2 = a;
                            }
                            S ^= (v[k] < 0.0f);
                        }
                        float m1c = corr_f32(&corr, m1), m2c = corr_f32(&corr, m2);
                        for (int k = 0; k < d; ++k) {
                            float mag = (k == idx) ? m2c : m1c;
                            c2v[(e0 + k) * Z + i] = (S ^ (v[k] < 0.0f)) ? -mag : mag;
                        }
                    }
                }
            }
            /* posteriors L_v = L_b + sum_k L_c->v^k (Sec. III) */
            for (int j = 0; j < N; ++j)
                Lv[j] = Lb[j];
            for (int e = 0; e < g.E; ++e)
                for (int i = 0; i < Z; ++i)
                    Lv[var_of(&g, e, i)] += c2v[e * Z + i];
            if (early_stop && syndrome_weight_f(&g, Lv) == 0) {
                done = t;
                break;
            }
        }
        for (int j = 0; j < K; ++j)
            bits[(size_t)b * K + j] = (Lv[j] < 0.0f);
        iters[b] = done;
        if (post)
            memcpy(post + (size_t)b * N, Lv, sizeof(float) * N);
    }
    free(Lb); free(Lv); free(c2v); free(v); free(tv);
    graph_free(&g);
    return OR_OK;
}

/* number of edges of the first n_rows rows (lets callers size the c2v buffers) */
int oracle_edge_count(const int16_t *base, int M_bg, int N_bg, int K_b, int Z, int n_rows)
{
    og_graph g;
    if (graph_build(base, M_bg, N_bg, K_b, Z, n_rows, &g) != OR_OK)
        return -1;
    int E = g.E;
    graph_free(&g);
    return E;
}

/* binary16 rounding, exported so the tests can pin it against numpy's float16 cast */
float oracle_round_half(double x)
{
    return round_half(x);
}

/* ------------------------------------------------- learned min-sum: forward and gradient
 *
 * Learned normalised-offset min-sum (an extension of the correction factor beta of
 * Sec. III to one (beta, gamma) pair per iteration t and base row r):
 *     m' = beta[t][r] * max(m - gamma[t][r], 0),  fp32 forward as in decode_one_f32.
 * Loss: mean over the batch and all used bits of the binary cross-entropy between
 * sigma(-L_v) (probability of bit 1) and the codeword bit:  softplus(-L) + c*L.
 * Gradient: reverse-mode through the unrolled layers.  For edge e of a check row with
 * v = L - c_old, c_new_e = s_e * beta * max(mag_e - gamma, 0), mag_e = min over the other
 * edges of |v| (m2 on the argmin edge, m1 elsewhere), s_e = sign product over the other
 * edges (treated as constant); the subgradient of mag_e goes to the edge attaining it
 * (lowest index on ties), d|v|/dv = sgn(v) with sgn(0) = +1, and d max(x, 0)/dx = [x > 0].
 * L_new = v + c_new.  Forward values of iteration t are recomputed from a checkpoint of
 * (L_v, c2v) taken at the start of t.  Computed in double.
 *
 * iter_weight (optional, [T]): the loss is sum_t iter_weight[t] * (BCE of the posteriors
 * after iteration t); NULL means the final posteriors only (weight 1 on t = T-1).  The
 * adjoint of the posteriors after iteration t then gains that term's gradient before
 * iteration t is undone.
 *
 * grad_params: [T][n_rows][2] (beta, gamma), summed over the decoded range.
 * grad_llr (optional): [batch][n_tx].  post (optional): [batch][N] final posteriors.
 * Returns the summed (not averaged) weighted loss over the range in *loss_sum.
 */
static double bce_term(double L, double c, double *grad)
{
    /* softplus(-L) + c L, computed stably; d/dL = c - sigma(-L) */
    const double sp = (L > 0 ? log1p(exp(-L)) : -L + log1p(exp(L)));
    *grad = c - 1.0 / (1.0 + exp(L));
    return sp + c * L;
}

int oracle_learned_grad(const int16_t *base, int M_bg, int N_bg, int K_b, int Z, int n_rows,
                        int punct, int n_tx, const float *params, int T, const float *llr,
                        const uint8_t *cw_bits, int cw_begin, int cw_end, double scale,
                        const double *iter_weight, double *grad_params, double *grad_llr,
                        float *post, double *loss_sum)
{
    og_graph g;
    int st = graph_build(base, M_bg, N_bg, K_b, Z, n_rows, &g);
    if (st != OR_OK)
        return st;
    const int N = g.n_cols * Z, EZ = g.E * Z;
    const int dmax = dec_max_degree(&g);
    float *Lv = (float *)malloc(sizeof(float) * N);
    float *c2v = (float *)malloc(sizeof(float) * (EZ + 1));
    float *ckL = (float *)malloc(sizeof(float) * (size_t)N * T);
    float *ckC = (float *)malloc(sizeof(float) * (size_t)(EZ + 1) * T);
    float *V = (float *)malloc(sizeof(float) * (EZ + 1));       /* v of every edge, one iteration */
    double *gL = (double *)malloc(sizeof(double) * N);
    double *gc = (double *)malloc(sizeof(double) * (EZ + 1));
    double *gv = (double *)malloc(sizeof(double) * (dmax + 1));
    if (!Lv || !c2v || !ckL || !ckC || !V || !gL || !gc || !gv) {
        free(Lv); free(c2v); free(ckL); free(ckC); free(V); free(gL); free(gc); free(gv);
        graph_free(&g);
        return OR_NO_MEM;
    }
    *loss_sum = 0.0;
    for (int b = cw_begin; b < cw_end; ++b) {
        /* forward with checkpoints */
        for (int j = 0; j < N; ++j)
            Lv[j] = 0.0f;
        for (int j = 0; j < n_tx; ++j)
            Lv[punct * Z + j] = llr[(size_t)b * n_tx + j];
        for (int k = 0; k < EZ; ++k)
            c2v[k] = 0.0f;
        for (int t = 0; t < T; ++t) {
            memcpy(ckL + (size_t)t * N, Lv, sizeof(float) * N);
            memcpy(ckC + (size_t)t * EZ, c2v, sizeof(float) * EZ);
            for (int r = 0; r < g.n_rows; ++r) {
                const float beta = params[(t * g.n_rows + r) * 2 + 0];
                const float gamma = params[(t * g.n_rows + r) * 2 + 1];
                const int e0 = g.row_ptr[r], d = g.row_ptr[r + 1] - e0;
                for (int i = 0; i < Z; ++i) {
                    float m1 = INFINITY, m2 = INFINITY;
                    int idx = -1, S = 0;
                    for (int k = 0; k < d; ++k) {
                        const float v = Lv[var_of(&g, e0 + k, i)] - c2v[(e0 + k) * Z + i];
                        V[(e0 + k) * Z + i] = v;
                        const float a = fabsf(v);
                        if (a < m1) {
                            m2 = m1;
                            m1 = a;
                            idx = k;
                        } else if (a < m2) {
                            m2 = a;
                        }
                        S ^= (v < 0.0f);
                    }
                    for (int k = 0; k < d; ++k) {
                        const float v = V[(e0 + k) * Z + i];
                        const float mag = (k == idx) ? m2 : m1;
                        float tm = mag - gamma;
                        tm = tm > 0.0f ? tm : 0.0f;
                        const float mc = beta * tm;
                        const float cv = (S ^ (v < 0.0f)) ? -mc : mc;
                        c2v[(e0 + k) * Z + i] = cv;
                        Lv[var_of(&g, e0 + k, i)] = v + cv;
                    }
                }
            }
        }
        if (post)
            memcpy(post + (size_t)b * N, Lv, sizeof(float) * N);
        /* loss term of the final posteriors and its gradient */
        const double w_last = iter_weight ? iter_weight[T - 1] : 1.0;
        for (int j = 0; j < N; ++j) {
            double gj;
            *loss_sum += w_last * bce_term(Lv[j], cw_bits[(size_t)b * N + j] & 1, &gj);
            gL[j] = scale * w_last * gj;
        }
        for (int k = 0; k < EZ; ++k)
            gc[k] = 0.0;
        /* reverse sweep over iterations */
        for (int t = T - 1; t >= 0; --t) {
            /* loss term of the posteriors after iteration t (< T-1): the checkpoint of t+1 */
            if (iter_weight && t < T - 1 && iter_weight[t] != 0.0)
                for (int j = 0; j < N; ++j) {
                    double gj;
                    *loss_sum += iter_weight[t] *
                                 bce_term(ckL[(size_t)(t + 1) * N + j],
                                          cw_bits[(size_t)b * N + j] & 1, &gj);
                    gL[j] += scale * iter_weight[t] * gj;
                }
            /* recompute the forward of iteration t from its checkpoint, keeping every v */
            memcpy(Lv, ckL + (size_t)t * N, sizeof(float) * N);
            memcpy(c2v, ckC + (size_t)t * EZ, sizeof(float) * EZ);
            for (int r = 0; r < g.n_rows; ++r) {
                const float beta = params[(t * g.n_rows + r) * 2 + 0];
                const float gamma = params[(t * g.n_rows + r) * 2 + 1];
                const int e0 = g.row_ptr[r], d = g.row_ptr[r + 1] - e0;
                for (int i = 0; i < Z; ++i) {
                    float m1 = INFINITY, m2 = INFINITY;
                    int idx = -1, S = 0;
                    for (int k = 0; k < d; ++k) {
                        const float v = Lv[var_of(&g, e0 + k, i)] - c2v[(e0 + k) * Z + i];
                        V[(e0 + k) * Z + i] = v;
                        const float a = fabsf(v);
                        if (a < m1) {
                            m2 = m1;
                            m1 = a;
                            idx = k;
                        } else if (a < m2) {
                            m2 = a;
                        }
                        S ^= (v < 0.0f);
                    }
                    for (int k = 0; k < d; ++k) {
                        const float v = V[(e0 + k) * Z + i];
                        const float mag = (k == idx) ? m2 : m1;
                        float tm = mag - gamma;
                        tm = tm > 0.0f ? tm : 0.0f;
                        const float mc = beta * tm;
                        const float cv = (S ^ (v < 0.0f)) ? -mc : mc;
                        Lv[var_of(&g, e0 + k, i)] = v + cv;
                        c2v[(e0 + k) * Z + i] = cv;
                    }
                }
            }
            /* backward through the layers of iteration t, last layer first */
            for (int r = g.n_rows - 1; r >= 0; --r) {
                const double beta = params[(t * g.n_rows + r) * 2 + 0];
                const double gamma = params[(t * g.n_rows + r) * 2 + 1];
                const int e0 = g.row_ptr[r], d = g.row_ptr[r + 1] - e0;
                double gb = 0.0, gg = 0.0;
                for (int i = 0; i < Z; ++i) {
                    /* row quantities from the stored v */
                    float m1 = INFINITY, m2 = INFINITY;
                    int idx = -1, idx2 = -1, S = 0;
                    for (int k = 0; k < d; ++k) {
                        const float a = fabsf(V[(e0 + k) * Z + i]);
                        if (a < m1) {
                            m2 = m1;
                            idx2 = idx;
                            m1 = a;
                            idx = k;
                        } else if (a < m2) {
                            m2 = a;
                            idx2 = k;
                        }
                        S ^= (V[(e0 + k) * Z + i] < 0.0f);
                    }
                    for (int k = 0; k < d; ++k)
                        gv[k] = gL[var_of(&g, e0 + k, i)];      /* dL_new / dv = 1 */
                    for (int k = 0; k < d; ++k) {
                        const float v = V[(e0 + k) * Z + i];
                        const double s = (S ^ (v < 0.0f)) ? -1.0 : 1.0;
                        const double mag = (k == idx) ? m2 : m1;
                        const double gcn = gL[var_of(&g, e0 + k, i)] + gc[(e0 + k) * Z + i];
                        const double act = mag - gamma > 0.0 ? 1.0 : 0.0;
                        gb += gcn * s * (mag - gamma > 0.0 ? mag - gamma : 0.0);
                        gg += -gcn * s * beta * act;
                        const double gmag = gcn * s * beta * act;
                        const int src = (k == idx) ? idx2 : idx;   /* edge attaining mag */
                        if (src >= 0 && gmag != 0.0) {
                            const float vs = V[(e0 + src) * Z + i];
                            gv[src] += gmag * (vs < 0.0f ? -1.0 : 1.0);
                        }
                    }
                    for (int k = 0; k < d; ++k) {
                        gL[var_of(&g, e0 + k, i)] = gv[k];       /* dv / dL_old = 1 */
                        gc[(e0 + k) * Z + i] = -gv[k];           /* dv / dc_old = -1 */
                    }
                }
                grad_params[(t * g.n_rows + r) * 2 + 0] += gb;
                grad_params[(t * g.n_rows + r) * 2 + 1] += gg;
            }
        }
        if (grad_llr)
            for (int j = 0; j < n_tx; ++j)
                grad_llr[(size_t)b * n_tx + j] = gL[punct * Z + j];
    }
    free(Lv); free(c2v); free(ckL); free(ckC); free(V); free(gL); free(gc); free(gv);
    graph_free(&g);
    return OR_OK;
}

/*
 * Seeded synthetic relations for the blocking workloads.
 *
 * This file generates input data only: random strings, skewed categorical
 * keys, lognormal numerics and near-duplicate copies made by random byte
 * edits and word swaps.  It holds none of the blocking method's arithmetic
 * (no predicate, rule, similarity or planning code), so that both the CPU
 * oracle and the GPU library can be fed from it without sharing code.
 *
 * Randomness: splitmix64 (Steele, Lea, Flood 2014), one sequential stream per
 * table.  Integer draws are bit-identical on every platform; floating-point
 * draws go through libm (log, cos, exp) and may differ in the last ulp between
 * C libraries, so expected values are always recomputed on the machine that
 * runs a test.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    SYN_LETTERS = 0,     /* a-z, length U[lo,hi] */
    SYN_WORDS = 1,       /* words of 3-12 letters split by one space, total length U[lo,hi] */
    SYN_ZIPF_INT = 2,    /* int32 categorical, Zipf(s) over card values */
    SYN_ZIPF_STR = 3,    /* string categorical, Zipf(s) over card values */
    SYN_UNIFORM_INT = 4, /* int32 categorical, uniform over card values */
    SYN_UNIFORM_STR = 5, /* string categorical, uniform over card values */
    SYN_LOGNORMAL = 6,   /* fp32 exp(N(mu, sigma)) */
    SYN_ROWID = 7        /* int32 row id after shuffling */
};

typedef struct {
    int32_t kind;
    int32_t lo, hi;     /* string length range */
    int64_t card;       /* categorical cardinality */
    double zipf_s;      /* Zipf exponent */
    double mu, sigma;   /* lognormal parameters */
    double null_rate;   /* probability that a row is missing (valid = 0) */
    int32_t edit;       /* near-duplicate copies edit this column */
    int32_t pad;
} syn_colspec;

typedef struct {
    int64_t n_rows;
    double dup_rate;      /* fraction of rows that copy an earlier row of this table */
    double cross_rate;    /* fraction of rows that copy a row of the source table */
    int32_t edit_lo, edit_hi;
    double swap_p;        /* probability of swapping two words in an edited string */
    double noise_rel;     /* fp32 copies get += N(0, noise_rel * |v|) */
    uint64_t seed;
    int32_t n_cols;
    int32_t shuffle;
} syn_tablespec;

/* One generated column.  Strings: bytes + n+1 offsets; int32/fp32: values. */
typedef struct {
    int32_t type;         /* 0 string, 1 int32, 2 fp32 */
    int32_t pad;
    int64_t n;
    uint8_t *bytes;
    uint64_t nbytes;
    uint32_t *off;
    int32_t *i32;
    float *f32;
    uint8_t *valid;       /* one byte per row, 1 = present */
} syn_col;

typedef struct { uint64_t s; } rng_t;

static uint64_t sm64(rng_t *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double u01(rng_t *r) { return (double)(sm64(r) >> 11) * (1.0 / 9007199254740992.0); }
static uint32_t below(rng_t *r, uint32_t n) {
    return (uint32_t)(((unsigned __int128)sm64(r) * n) >> 64);
}
static double normal(rng_t *r) {
    double u1 = u01(r), u2 = u01(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* ---- growable byte buffer for string columns ---- */
typedef struct { uint8_t *p; uint64_t n, cap; } buf_t;
static int buf_reserve(buf_t *b, uint64_t extra) {
    if (b->n + extra <= b->cap) return 0;
    uint64_t cap = b->cap ? b->cap : 4096;
    while (cap < b->n + extra) cap *= 2;
    uint8_t *p = (uint8_t *)realloc(b->p, cap);
    if (!p) return -1;
    b->p = p; b->cap = cap;
    return 0;
}

/* ---- categorical support ---- */
typedef struct { double *cdf; int64_t card; uint32_t *perm; int width; } cat_t;

static int cat_init(cat_t *c, const syn_colspec *cs, rng_t *r) {
    c->card = cs->card > 0 ? cs->card : 1;
    c->cdf = NULL;
    if (cs->kind == SYN_ZIPF_INT || cs->kind == SYN_ZIPF_STR) {
        c->cdf = (double *)malloc(sizeof(double) * (size_t)c->card);
        if (!c->cdf) return -1;
        double acc = 0;
        for (int64_t i = 0; i < c->card; i++) { acc += pow((double)(i + 1), -cs->zipf_s); c->cdf[i] = acc; }
        for (int64_t i = 0; i < c->card; i++) c->cdf[i] /= acc;
    }
    /* value ids are a random permutation of ranks, so the code does not reveal frequency */
    c->perm = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)c->card);
    if (!c->perm) return -1;
    for (int64_t i = 0; i < c->card; i++) c->perm[i] = (uint32_t)i;
    for (int64_t i = c->card - 1; i > 0; i--) {
        uint32_t j = below(r, (uint32_t)(i + 1));
        uint32_t t = c->perm[i]; c->perm[i] = c->perm[j]; c->perm[j] = t;
    }
    c->width = 1;
    for (int64_t v = 26; v < c->card; v *= 26) c->width++;
    return 0;
}
static void cat_free(cat_t *c) { free(c->cdf); free(c->perm); }
static uint32_t cat_draw(cat_t *c, rng_t *r) {
    uint32_t rank;
    if (c->cdf) {
        double u = u01(r);
        int64_t lo = 0, hi = c->card - 1;
        while (lo < hi) { int64_t mid = (lo + hi) / 2; if (c->cdf[mid] < u) lo = mid + 1; else hi = mid; }
        rank = (uint32_t)lo;
    } else {
        rank = below(r, (uint32_t)c->card);
    }
    return c->perm[rank];
}

/* ---- string makers ---- */
static int put_letters(buf_t *b, rng_t *r, int len) {
    if (buf_reserve(b, (uint64_t)len)) return -1;
    for (int i = 0; i < len; i++) b->p[b->n++] = (uint8_t)('a' + below(r, 26));
    return 0;
}
static int put_words(buf_t *b, rng_t *r, int len) {
    if (buf_reserve(b, (uint64_t)len)) return -1;
    int w = 0;
    uint64_t start = b->n;
    while (w < len) {
        if (w > 0) { b->p[b->n++] = ' '; w++; if (w >= len) break; }
        int wl = 3 + (int)below(r, 10);
        for (int i = 0; i < wl && w < len; i++, w++) b->p[b->n++] = (uint8_t)('a' + below(r, 26));
    }
    if (b->n > start && b->p[b->n - 1] == ' ') b->p[b->n - 1] = (uint8_t)('a' + below(r, 26));
    return 0;
}
static int put_catstr(buf_t *b, uint32_t v, int width) {
    if (buf_reserve(b, (uint64_t)width + 1)) return -1;
    b->p[b->n++] = 'k';
    for (int i = 0; i < width; i++) { b->p[b->n++] = (uint8_t)('a' + v % 26); v /= 26; }
    return 0;
}

/* copy src[0..len) into b with word swap and 1..k random byte edits */
static int put_edited(buf_t *b, rng_t *r, const uint8_t *src, uint32_t len, const syn_tablespec *ts) {
    uint32_t cap = len + (uint32_t)ts->edit_hi + 8;
    uint8_t *tmp = (uint8_t *)malloc(cap), *tmp2 = (uint8_t *)malloc(cap);
    if (!tmp || !tmp2) { free(tmp); free(tmp2); return -1; }
    memcpy(tmp, src, len);
    uint32_t n = len;
    if (ts->swap_p > 0 && u01(r) < ts->swap_p) {
        /* word boundaries */
        uint32_t ws[64], we[64]; int nw = 0; uint32_t i = 0;
        while (i < n && nw < 64) {
            while (i < n && tmp[i] == ' ') i++;
            if (i >= n) break;
            ws[nw] = i;
            while (i < n && tmp[i] != ' ') i++;
            we[nw++] = i;
        }
        if (nw >= 2) {
            int a = (int)below(r, (uint32_t)nw), c = (int)below(r, (uint32_t)(nw - 1));
            if (c >= a) c++;
            if (a > c) { int t = a; a = c; c = t; }
            /* rebuild: [0,ws[a]) + word c + [we[a],ws[c]) + word a + [we[c],n) */
            uint32_t o = 0;
            memcpy(tmp2 + o, tmp, ws[a]); o += ws[a];
            memcpy(tmp2 + o, tmp + ws[c], we[c] - ws[c]); o += we[c] - ws[c];
            memcpy(tmp2 + o, tmp + we[a], ws[c] - we[a]); o += ws[c] - we[a];
            memcpy(tmp2 + o, tmp + ws[a], we[a] - ws[a]); o += we[a] - ws[a];
            memcpy(tmp2 + o, tmp + we[c], n - we[c]); o += n - we[c];
            memcpy(tmp, tmp2, o); n = o;
        }
    }
    int k = ts->edit_lo + (int)below(r, (uint32_t)(ts->edit_hi - ts->edit_lo + 1));
    for (int e = 0; e < k; e++) {
        uint32_t op = below(r, 3);
        if (op == 1 && n <= 1) op = 0;
        if (op == 0) {               /* insert */
            uint32_t pos = below(r, n + 1);
            memmove(tmp + pos + 1, tmp + pos, n - pos);
            tmp[pos] = (uint8_t)('a' + below(r, 26)); n++;
        } else if (op == 1) {        /* delete */
            uint32_t pos = below(r, n);
            memmove(tmp + pos, tmp + pos + 1, n - pos - 1); n--;
        } else if (n > 0) {          /* substitute */
            uint32_t pos = below(r, n);
            tmp[pos] = (uint8_t)('a' + below(r, 26));
        }
    }
    int rc = buf_reserve(b, n);
    if (!rc) { memcpy(b->p + b->n, tmp, n); b->n += n; }
    free(tmp); free(tmp2);
    return rc;
}

void syn_free_cols(syn_col *cols, int32_t n_cols) {
    for (int c = 0; c < n_cols; c++) {
        free(cols[c].bytes); free(cols[c].off); free(cols[c].i32); free(cols[c].f32); free(cols[c].valid);
        memset(&cols[c], 0, sizeof(syn_col));
    }
}

/*
 * Generate one table.  `src` (optional, n_src rows with the same schema)
 * is the table that cross-duplicates copy from.  Returns 0 or -1 (OOM).
 */
int syn_make_table(const syn_tablespec *ts, const syn_colspec *cs, const syn_col *src, int64_t n_src,
                   syn_col *out) {
    rng_t r = { ts->seed * 0x2545F4914F6CDD1Dull + 0x1234567ull };
    const int64_t n = ts->n_rows;
    const int nc = ts->n_cols;
    int64_t n_cross = (src && n_src > 0) ? (int64_t)llround((double)n * ts->cross_rate) : 0;
    int64_t n_dup = (int64_t)llround((double)n * ts->dup_rate);
    if (n_cross + n_dup > n) n_dup = n - n_cross;
    int64_t n_fresh = n - n_cross - n_dup;
    if (n_fresh < 1 && n_dup > 0) { n_fresh = 1; n_dup = n - n_cross - 1; }

    /* origin of every row before shuffling: -1 fresh, >=0 copy of row (this table), <=-2 copy of src row -(v+2) */
    int64_t *origin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    cat_t *cats = (cat_t *)calloc((size_t)nc, sizeof(cat_t));
    buf_t *bufs = (buf_t *)calloc((size_t)nc, sizeof(buf_t));
    uint32_t **offs = (uint32_t **)calloc((size_t)nc, sizeof(uint32_t *));
    if (!origin || !perm || !cats || !bufs || !offs) goto oom;

    for (int64_t i = 0; i < n; i++) {
        if (i < n_fresh) origin[i] = -1;
        else if (i < n_fresh + n_dup) origin[i] = (int64_t)below(&r, (uint32_t)n_fresh);
        else origin[i] = -2 - (int64_t)below(&r, (uint32_t)n_src);
    }
    for (int64_t i = 0; i < n; i++) perm[i] = i;
    if (ts->shuffle)
        for (int64_t i = n - 1; i > 0; i--) {
            int64_t j = (int64_t)below(&r, (uint32_t)(i + 1));
            int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }

    for (int c = 0; c < nc; c++) {
        const syn_colspec *s = &cs[c];
        syn_col *o = &out[c];
        memset(o, 0, sizeof(*o));
        o->n = n;
        o->valid = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
        if (!o->valid) goto oom;
        int is_str = (s->kind == SYN_LETTERS || s->kind == SYN_WORDS || s->kind == SYN_ZIPF_STR ||
                      s->kind == SYN_UNIFORM_STR);
        int is_cat = (s->kind == SYN_ZIPF_INT || s->kind == SYN_ZIPF_STR || s->kind == SYN_UNIFORM_INT ||
                      s->kind == SYN_UNIFORM_STR);
        if (is_cat && cat_init(&cats[c], s, &r)) goto oom;
        o->type = is_str ? 0 : (s->kind == SYN_LOGNORMAL ? 2 : 1);
        if (is_str) {
            offs[c] = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
            if (!offs[c]) goto oom;
            offs[c][0] = 0;
        } else if (o->type == 1) {
            o->i32 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            if (!o->i32) goto oom;
        } else {
            o->f32 = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
            if (!o->f32) goto oom;
        }
    }

    /* generate rows in origin order (copies always refer to earlier fresh rows) */
    for (int64_t i = 0; i < n; i++) {
        for (int c = 0; c < nc; c++) {
            const syn_colspec *s = &cs[c];
            syn_col *o = &out[c];
            int64_t org = origin[i];
            const syn_col *from = NULL; int64_t fi = -1;
            if (org >= 0) { from = o; fi = org; }
            else if (org <= -2) { from = &src[c]; fi = -2 - org; }
            uint8_t v = 1;
            if (from) v = from->valid[fi];
            else if (s->null_rate > 0 && u01(&r) < s->null_rate) v = 0;
            o->valid[i] = v;
            if (o->type == 0) {
                buf_t *b = &bufs[c];
                int rc = 0;
                if (from) {
                    const uint8_t *sp = (from == o) ? b->p + offs[c][fi] : from->bytes + from->off[fi];
                    uint32_t sl = (from == o) ? offs[c][fi + 1] - offs[c][fi] : from->off[fi + 1] - from->off[fi];
                    if (s->edit && v) {
                        /* copy out first: the buffer may move while growing */
                        uint8_t *cp = (uint8_t *)malloc(sl + 1);
                        if (!cp) goto oom;
                        memcpy(cp, sp, sl);
                        rc = put_edited(b, &r, cp, sl, ts);
                        free(cp);
                    } else {
                        uint8_t *cp = (uint8_t *)malloc(sl + 1);
                        if (!cp) goto oom;
                        memcpy(cp, sp, sl);
                        rc = buf_reserve(b, sl);
                        if (!rc) { memcpy(b->p + b->n, cp, sl); b->n += sl; }
                        free(cp);
                    }
                } else if (v) {
                    int len = s->lo + (int)below(&r, (uint32_t)(s->hi - s->lo + 1));
                    if (s->kind == SYN_LETTERS) rc = put_letters(b, &r, len);
                    else if (s->kind == SYN_WORDS) rc = put_words(b, &r, len);
                    else rc = put_catstr(b, cat_draw(&cats[c], &r), cats[c].width);
                }
                if (rc) goto oom;
                if (b->n > 0xFFFFFFFFull) goto oom;
                offs[c][i + 1] = (uint32_t)b->n;
            } else if (o->type == 1) {
                int32_t x = 0;
                if (from) x = (from == o) ? o->i32[fi] : from->i32[fi];
                else if (s->kind == SYN_ROWID) x = 0;
                else if (v) x = (int32_t)cat_draw(&cats[c], &r);
                o->i32[i] = x;
            } else {
                float x = 0.f;
                if (from) {
                    x = (from == o) ? o->f32[fi] : from->f32[fi];
                    if (s->edit && v && ts->noise_rel > 0)
                        x = (float)((double)x + normal(&r) * ts->noise_rel * fabs((double)x));
                } else if (v) {
                    x = (float)exp(s->mu + s->sigma * normal(&r));
                }
                o->f32[i] = x;
            }
        }
    }

    /* apply the row permutation: final row perm[i] <- generated row i */
    for (int c = 0; c < nc; c++) {
        syn_col *o = &out[c];
        uint8_t *valid = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
        if (!valid) goto oom;
        for (int64_t i = 0; i < n; i++) valid[perm[i]] = o->valid[i];
        if (o->type == 0) {
            uint32_t *off = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
            uint8_t *bytes = (uint8_t *)malloc(bufs[c].n > 0 ? bufs[c].n : 1);
            if (!off || !bytes) { free(off); free(bytes); free(valid); goto oom; }
            /* lengths in final order, then prefix sum, then copy */
            int64_t *inv = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
            if (!inv) { free(off); free(bytes); free(valid); goto oom; }
            for (int64_t i = 0; i < n; i++) inv[perm[i]] = i;
            off[0] = 0;
            for (int64_t j = 0; j < n; j++) {
                int64_t i = inv[j];
                off[j + 1] = off[j] + (offs[c][i + 1] - offs[c][i]);
            }
            for (int64_t j = 0; j < n; j++) {
                int64_t i = inv[j];
                memcpy(bytes + off[j], bufs[c].p + offs[c][i], offs[c][i + 1] - offs[c][i]);
            }
            free(inv);
            o->bytes = bytes; o->nbytes = bufs[c].n; o->off = off;
            free(bufs[c].p); bufs[c].p = NULL;
            free(offs[c]); offs[c] = NULL;
        } else if (o->type == 1) {
            int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
            if (!x) { free(valid); goto oom; }
            for (int64_t i = 0; i < n; i++) x[perm[i]] = o->i32[i];
            if (cs[c].kind == SYN_ROWID) for (int64_t i = 0; i < n; i++) x[i] = (int32_t)i;
            free(o->i32); o->i32 = x;
        } else {
            float *x = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
            if (!x) { free(valid); goto oom; }
            for (int64_t i = 0; i < n; i++) x[perm[i]] = o->f32[i];
            free(o->f32); o->f32 = x;
        }
        free(o->valid); o->valid = valid;
    }

    for (int c = 0; c < nc; c++) { cat_free(&cats[c]); free(bufs[c].p); free(offs[c]); }
    free(cats); free(bufs); free(offs); free(origin); free(perm);
    return 0;
oom:
    if (cats) for (int c = 0; c < nc; c++) cat_free(&cats[c]);
    if (bufs) for (int c = 0; c < nc; c++) free(bufs[c].p);
    if (offs) for (int c = 0; c < nc; c++) free(offs[c]);
    free(cats); free(bufs); free(offs); free(origin); free(perm);
    syn_free_cols(out, nc);
    return -1;
}

/* 64-bit draw for callers that need extra seeded choices (e.g. rule sets) */
uint64_t syn_mix(uint64_t seed, uint64_t k) {
    rng_t r = { seed ^ (k * 0xD1B54A32D192ED03ull) };
    return sm64(&r);
}

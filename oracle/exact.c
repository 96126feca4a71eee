/*
 * Exact sign of a sum of products of doubles, by plain big-integer arithmetic.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper decides every geometric test exactly (Sec. 7: exact arithmetic,
 * simulation of simplicity).  The oracle's exact path makes no use of
 * floating-point expansions: every double is split into an integer
 * mantissa m (< 2^53) and a power of two, each monomial becomes an integer
 * times 2^e, all monomials are aligned to the smallest exponent, and the
 * positive and negative parts are summed in two unsigned big integers that
 * are finally compared.  Slow and obviously exact.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LIMB_BITS 32
/* Any degree-4 monomial of doubles spans < 4*2098+212 bits, i.e. < 270 limbs. */
#define MAX_LIMBS 300

typedef struct {
    uint32_t w[10];    /* little-endian limbs of |product of mantissas| */
    int nw;            /* used limbs */
    int e;             /* value = w * 2^e */
    int sign;
} bigmono;

/* w (nw limbs) *= m (an integer < 2^64), schoolbook, in place */
static void mul_small(uint32_t* w, int* nw, uint64_t m) {
    uint32_t mm[2] = {(uint32_t)(m & 0xffffffffu), (uint32_t)(m >> 32)};
    uint32_t out[10];
    memset(out, 0, sizeof(out));
    for (int i = 0; i < *nw; ++i) {
        uint64_t carry = 0;
        for (int j = 0; j < 2; ++j) {
            uint64_t t = (uint64_t)w[i] * mm[j] + out[i + j] + carry;
            out[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        for (int k = i + 2; carry; ++k) {
            uint64_t t = (uint64_t)out[k] + carry;
            out[k] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    int n = *nw + 2;
    while (n > 1 && out[n - 1] == 0) --n;
    memcpy(w, out, sizeof(out));
    *nw = n;
}

/* Decompose x != 0 into (mantissa, exponent) with |x| = mant * 2^exp. */
static void split_double(double x, uint64_t* mant, int* ex) {
    int e;
    double fr = frexp(fabs(x), &e);         /* fr in [0.5, 1) */
    *mant = (uint64_t)ldexp(fr, 53);        /* exact: fr has <= 53 significant bits */
    *ex = e - 53;
}

static int bitlen(const bigmono* b) {
    int top = b->nw - 1;
    uint32_t v = b->w[top];
    int n = 0;
    while (v) { ++n; v >>= 1; }
    return top * LIMB_BITS + n;
}

/* acc (nl limbs) += b * 2^shift */
static void add_shifted(uint32_t* acc, int nl, const bigmono* b, int shift) {
    int ws = shift / LIMB_BITS, bs = shift % LIMB_BITS;
    uint64_t carry = 0;
    for (int i = 0; i <= b->nw; ++i) {
        uint32_t cur = (i < b->nw) ? b->w[i] : 0;
        uint32_t prev = (i > 0) ? b->w[i - 1] : 0;
        uint32_t part = bs ? (uint32_t)((cur << bs) | (prev >> (LIMB_BITS - bs))) : cur;
        uint64_t t = (uint64_t)acc[ws + i] + part + carry;
        acc[ws + i] = (uint32_t)t;
        carry = t >> 32;
    }
    for (int j = ws + b->nw + 1; carry && j < nl; ++j) {
        uint64_t t = (uint64_t)acc[j] + carry;
        acc[j] = (uint32_t)t;
        carry = t >> 32;
    }
}

int or_exact_sign(const or_mono* m, int n) {
    bigmono stack_bm[64];
    bigmono* bm = n <= 64 ? stack_bm : (bigmono*)malloc(sizeof(bigmono) * (size_t)n);
    int nb = 0;
    for (int i = 0; i < n; ++i) {
        int zero = 0, sign = m[i].sign, e = 0;
        bigmono b;
        memset(&b, 0, sizeof(b));
        b.w[0] = 1;
        b.nw = 1;
        for (int k = 0; k < m[i].k; ++k) {
            double x = m[i].f[k];
            if (x == 0.0) { zero = 1; break; }
            if (x < 0) sign = -sign;
            uint64_t mant;
            int ex;
            split_double(x, &mant, &ex);
            mul_small(b.w, &b.nw, mant);
            e += ex;
        }
        if (zero || sign == 0) continue;
        b.e = e;
        b.sign = sign;
        bm[nb++] = b;
    }
    if (nb == 0) { if (bm != stack_bm) free(bm); return 0; }
    int emin = bm[0].e, etop = 0;
    for (int i = 0; i < nb; ++i) if (bm[i].e < emin) emin = bm[i].e;
    for (int i = 0; i < nb; ++i) {
        int t = bm[i].e - emin + bitlen(&bm[i]);
        if (t > etop) etop = t;
    }
    /* + log2(n) carry bits + slack */
    int nl = etop / LIMB_BITS + 4;
    int cb = 0;
    while ((1 << cb) < nb) ++cb;
    nl += cb / LIMB_BITS + 1;
    uint32_t pos_s[MAX_LIMBS], neg_s[MAX_LIMBS];
    uint32_t *pos = pos_s, *neg = neg_s;
    if (nl > MAX_LIMBS) {
        pos = (uint32_t*)calloc((size_t)nl, sizeof(uint32_t));
        neg = (uint32_t*)calloc((size_t)nl, sizeof(uint32_t));
    } else {
        memset(pos, 0, sizeof(uint32_t) * (size_t)nl);
        memset(neg, 0, sizeof(uint32_t) * (size_t)nl);
    }
    for (int i = 0; i < nb; ++i)
        add_shifted(bm[i].sign > 0 ? pos : neg, nl, &bm[i], bm[i].e - emin);
    int s = 0;
    for (int i = nl - 1; i >= 0; --i) {
        if (pos[i] != neg[i]) { s = pos[i] > neg[i] ? 1 : -1; break; }
    }
    if (pos != pos_s) { free(pos); free(neg); }
    if (bm != stack_bm) free(bm);
    return s;
}

/*
 * psl_oracle.c -- plain, slow CPU oracle for the two-phase low-PSL search of
 * Boskovic and Brest, "Two-phase Optimization of Binary Sequences with Low
 * Peak Sidelobe Level Value" (arXiv 2107.09801).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file; the CUDA library never does, and the
 * two share no code, header, table or helper.
 *
 * What it follows, passage by passage:
 *   Eq. (1)   a sequence is s_0..s_{L-1}, each +1 or -1 (0-based here).
 *   Eq. (2)   C_k = sum_{i=0}^{L-1-k} s_i s_{i+k},  k = 0..L-1.
 *   Eq. (3)   PSL = max |C_k| over the sidelobes.  The printed range
 *             "1 < k < L" is read as k = 1..L-1, the range of Eq. (4).
 *   Eq. (4)   F_alpha = sum_{k=1}^{L-1} |C_k|^alpha, kept as an EXACT integer
 *             (384-bit two's complement) so that every "<", ">" and "=" of
 *             Algorithm 1 is decided exactly; the FP64 value reported is the
 *             correctly rounded exact value.  A naive ordered FP64 sum is also
 *             available for comparison.
 *   Sec. 3    one-element flip: flipping s_j changes C_k (k >= 1) by
 *             -2 s_j (s_{j+k} + s_{j-k}), a missing partner counting 0.
 *   Alg. 1    the search: random start, window of N_lmt neighbours starting
 *             after Rand() % L, forced move to the first minimum of F, best
 *             PSL tracked over every evaluated neighbour (first minimum),
 *             unimproved counter, phase switch after LS_lmt non-improving
 *             steps that perturbs local_best with FLIP_lmt flips and toggles
 *             alpha between alpha1 and alpha2.
 *
 * Readings where the paper is silent (listed again in the design notes):
 *   - Rand is SplitMix64 (Steele, Lea, Flood 2014): draw n of a walk with
 *     seed S is mix(S + (n+1) * 0x9E3779B97F4A7C15).  Draw order: ceil(L/64)
 *     draws for the start sequence (bit b of draw q gives s_{64q+b}, bit 1
 *     meaning -1); then one draw per step (start = draw % L); then, at a
 *     switch, draws % L until min(FLIP_lmt, L) distinct positions are found.
 *   - The window has N = min(N_lmt, L) neighbours j = (start + i) % L,
 *     i = 1..N, evaluated in that scan order.
 *   - psl_best / solution_best start as PSL(pivot_0) / pivot_0; local_best
 *     starts as pivot_0.  At a switch local_best is left unchanged.
 *   - The budget counts while-iterations; every iteration makes one move.
 *   - alpha is an integer in 1..16.
 *   - When alpha1 == alpha2 the objective never changes, so the lowest F over
 *     every pivot the walk visits (the start, each move, each perturbed pivot
 *     of a switch; the first one on ties) is kept with its sequence.  With
 *     alpha = 2 that F is the energy sum C_k^2 of the merit factor
 *     MF = L^2 / (2 sum C_k^2) defined in Sec. 2.  With alpha1 != alpha2 F
 *     values of the two phases are not comparable and nothing is kept past
 *     the start.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* 384-bit two's-complement integers (6 little-endian 64-bit limbs).         */
/* |C_k| < 2^20 and alpha <= 16 give |C_k|^alpha < 2^320; a sum of fewer    */
/* than 2^20 such terms stays below 2^340, far inside the signed range.      */
/* ------------------------------------------------------------------------ */
#define WL 6
typedef struct { uint64_t w[WL]; } wide_t;

static void wide_set_u64(wide_t *a, uint64_t v) {
    a->w[0] = v;
    for (int i = 1; i < WL; i++) a->w[i] = 0;
}

static void wide_add(wide_t *r, const wide_t *a, const wide_t *b) {
    unsigned __int128 carry = 0;
    for (int i = 0; i < WL; i++) {
        unsigned __int128 t = (unsigned __int128)a->w[i] + b->w[i] + carry;
        r->w[i] = (uint64_t)t;
        carry = t >> 64;
    }
}

static void wide_neg(wide_t *r, const wide_t *a) {
    wide_t one, inv;
    for (int i = 0; i < WL; i++) inv.w[i] = ~a->w[i];
    wide_set_u64(&one, 1);
    wide_add(r, &inv, &one);
}

static void wide_sub(wide_t *r, const wide_t *a, const wide_t *b) {
    wide_t nb;
    wide_neg(&nb, b);
    wide_add(r, a, &nb);
}

/* r = a * m for a non-negative a (no overflow for the ranges used here). */
static void wide_mul_u32(wide_t *r, const wide_t *a, uint32_t m) {
    unsigned __int128 carry = 0;
    for (int i = 0; i < WL; i++) {
        unsigned __int128 t = (unsigned __int128)a->w[i] * m + carry;
        r->w[i] = (uint64_t)t;
        carry = t >> 64;
    }
}

static int wide_is_neg(const wide_t *a) { return (int)(a->w[WL - 1] >> 63); }

static int wide_is_zero(const wide_t *a) {
    for (int i = 0; i < WL; i++)
        if (a->w[i]) return 0;
    return 1;
}

/* sign of a - b: -1, 0 or +1 */
static int wide_cmp(const wide_t *a, const wide_t *b) {
    wide_t d;
    wide_sub(&d, a, b);
    if (wide_is_zero(&d)) return 0;
    return wide_is_neg(&d) ? -1 : 1;
}

static int wide_bit(const wide_t *a, int i) { return (int)((a->w[i / 64] >> (i % 64)) & 1u); }

/* Correctly rounded (round-to-nearest, ties-to-even) conversion to double. */
static double wide_to_double(const wide_t *a) {
    wide_t m = *a;
    int neg = 0;
    if (wide_is_neg(&m)) {
        wide_neg(&m, &m);
        neg = 1;
    }
    int h = -1;
    for (int i = 64 * WL - 1; i >= 0; i--)
        if (wide_bit(&m, i)) {
            h = i;
            break;
        }
    if (h < 0) return 0.0;
    double r;
    if (h <= 52) {
        r = (double)m.w[0];
    } else {
        int drop = h - 52; /* bits below the 53-bit significand */
        uint64_t mant = 0;
        for (int i = h; i >= drop; i--) mant = (mant << 1) | (uint64_t)wide_bit(&m, i);
        int round = wide_bit(&m, drop - 1);
        int sticky = 0;
        for (int i = drop - 2; i >= 0; i--) sticky |= wide_bit(&m, i);
        if (round && (sticky || (mant & 1u))) mant++;
        r = ldexp((double)mant, drop);
    }
    return neg ? -r : r;
}

/* ------------------------------------------------------------------------ */
/* Rand: SplitMix64, counter form (reading of Rand in Alg. 1).               */
/* ------------------------------------------------------------------------ */
ORC_API uint64_t orc_splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Rand(L, SEED) of Alg. 1: the uniform +-1 start sequence, draws 0..ceil(L/64)-1. */
ORC_API void orc_init_seq(uint32_t L, uint64_t seed, int8_t *s) {
    for (uint32_t i = 0; i < L; i++) {
        uint64_t d = orc_splitmix64(seed, i / 64);
        s[i] = ((d >> (i % 64)) & 1u) ? -1 : 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. (2), Eq. (3), Eq. (4)                                                 */
/* ------------------------------------------------------------------------ */
ORC_API void orc_autocorr(const int8_t *s, uint32_t L, int32_t *C) {
    for (uint32_t k = 0; k < L; k++) {
        int32_t c = 0;
        for (uint32_t i = 0; i + k < L; i++) c += (int32_t)s[i] * (int32_t)s[i + k];
        C[k] = c;
    }
}

ORC_API int32_t orc_psl(const int32_t *C, uint32_t L) {
    int32_t p = 0;
    for (uint32_t k = 1; k < L; k++) {
        int32_t a = C[k] < 0 ? -C[k] : C[k];
        if (a > p) p = a;
    }
    return p;
}

/* P[c] = c^alpha for c = 0..cmax. */
static wide_t *power_table(uint32_t cmax, uint32_t alpha) {
    wide_t *P = (wide_t *)malloc(sizeof(wide_t) * ((size_t)cmax + 1));
    if (!P) return NULL;
    for (uint32_t c = 0; c <= cmax; c++) {
        wide_set_u64(&P[c], 1);
        for (uint32_t a = 0; a < alpha; a++) wide_mul_u32(&P[c], &P[c], c);
    }
    return P;
}

static uint32_t max_abs_sidelobe(const int32_t *C, uint32_t L) { return (uint32_t)orc_psl(C, L); }

/* Eq. (4) summed from a power table. */
static void fitness_exact_tab(const int32_t *C, uint32_t L, const wide_t *P, wide_t *F) {
    wide_set_u64(F, 0);
    for (uint32_t k = 1; k < L; k++) {
        uint32_t a = (uint32_t)(C[k] < 0 ? -C[k] : C[k]);
        wide_add(F, F, &P[a]);
    }
}

/* Eq. (4) as a naive FP64 sum in k order, |C_k|^alpha by repeated products. */
static double fitness_naive(const int32_t *C, uint32_t L, uint32_t alpha) {
    double f = 0.0;
    for (uint32_t k = 1; k < L; k++) {
        double a = fabs((double)C[k]), p = 1.0;
        for (uint32_t t = 0; t < alpha; t++) p *= a;
        f += p;
    }
    return f;
}

/* Eq. (4): exact value into limbs[6], its rounded FP64 value, and the naive sum. */
ORC_API int orc_fitness(const int32_t *C, uint32_t L, uint32_t alpha, uint64_t *limbs, double *f_rounded,
                        double *f_naive) {
    wide_t *P = power_table(max_abs_sidelobe(C, L), alpha);
    if (!P) return -1;
    wide_t F;
    fitness_exact_tab(C, L, P, &F);
    free(P);
    if (limbs) memcpy(limbs, F.w, sizeof F.w);
    if (f_rounded) *f_rounded = wide_to_double(&F);
    if (f_naive) *f_naive = fitness_naive(C, L, alpha);
    return 0;
}

/* Exposed so that tests can compare the rounding with another implementation. */
ORC_API double orc_wide_to_double(const uint64_t *limbs) {
    wide_t a;
    memcpy(a.w, limbs, sizeof a.w);
    return wide_to_double(&a);
}

/* Sec. 3, one-element flip: autocorrelation of the neighbour with s_j flipped. */
ORC_API void orc_flip_autocorr(const int8_t *s, const int32_t *C, uint32_t L, uint32_t j, int32_t *Cn) {
    Cn[0] = C[0];
    for (uint32_t k = 1; k < L; k++) {
        int32_t partners = 0;
        if (j + k < L) partners += s[j + k];
        if (j >= k) partners += s[j - k];
        Cn[k] = C[k] - 2 * (int32_t)s[j] * partners;
    }
}

/* ------------------------------------------------------------------------ */
/* Exhaustive minimum PSL (Eq. 5, goal of the problem) for tiny L.           */
/* s_0 = +1 is fixed: negating a sequence leaves every |C_k| unchanged.      */
/* ------------------------------------------------------------------------ */
ORC_API int32_t orc_brute_min_psl(uint32_t L, int8_t *best_seq) {
    if (L < 2 || L > 24) return -1;
    int8_t s[24];
    int32_t C[24];
    int32_t best = 1 << 30;
    uint64_t count = 1ULL << (L - 1);
    for (uint64_t m = 0; m < count; m++) {
        s[0] = 1;
        for (uint32_t i = 1; i < L; i++) s[i] = ((m >> (i - 1)) & 1u) ? -1 : 1;
        orc_autocorr(s, L, C);
        int32_t p = orc_psl(C, L);
        if (p < best) {
            best = p;
            if (best_seq) memcpy(best_seq, s, L);
        }
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t L, n_lmt, ls_lmt, flip_lmt, alpha1, alpha2;
    uint64_t seed;
} orc_params;

typedef struct {
    int8_t *s;          /* pivot (length L)                        */
    int8_t *local_best; /* local_best of Alg. 1 (length L)         */
    int8_t *sol_best;   /* solution_best of Alg. 1 (length L)      */
    int32_t *C;         /* C_0..C_{L-1} of the pivot              */
    uint64_t value_local[WL];
    uint64_t F[WL];     /* F_alpha(pivot), exact                   */
    uint32_t alpha, unimproved;
    int32_t psl, psl_best;
    uint64_t rng_ctr, steps, near_ties;
    int8_t *fbest_seq;  /* lowest-F pivot when alpha1 == alpha2      */
    uint64_t F_best[WL];
} orc_state;

typedef struct {
    uint64_t step;
    uint32_t start, kstar, alpha, unimproved;
    int32_t psl, psl_best, win_psl;
    uint32_t win_psl_j, flags, nflip;
    double value_step, value_naive;
    uint64_t value_exact[WL];
} orc_trace;

enum { ORC_IMPROVED = 1, ORC_WORSE = 2, ORC_SWITCH = 4, ORC_PSL_BEST = 8, ORC_NAIVE_DIFFERS = 16 };
enum { ORC_MODE_FULL = 1, ORC_MODE_CROSSCHECK = 2, ORC_MODE_NAIVE = 4 };

static int param_check(const orc_params *p) {
    if (p->L < 2 || p->L > (1u << 20) - 1) return -1;
    if (p->alpha1 < 1 || p->alpha1 > 16 || p->alpha2 < 1 || p->alpha2 > 16) return -1;
    if (p->n_lmt < 1) return -1;
    return 0;
}

/* Alg. 1: the initialisation before the search loop. */
ORC_API int orc_init(const orc_params *p, orc_state *st) {
    if (param_check(p)) return -1;
    uint32_t L = p->L;
    orc_init_seq(L, p->seed, st->s);
    orc_autocorr(st->s, L, st->C);
    memcpy(st->local_best, st->s, L);
    memcpy(st->sol_best, st->s, L);
    st->alpha = p->alpha1;
    uint64_t limbs[WL];
    if (orc_fitness(st->C, L, st->alpha, limbs, NULL, NULL)) return -1;
    memcpy(st->value_local, limbs, sizeof limbs);
    memcpy(st->F, limbs, sizeof limbs);
    memcpy(st->F_best, limbs, sizeof limbs);
    memcpy(st->fbest_seq, st->s, L);
    st->unimproved = 0;
    st->psl = orc_psl(st->C, L);
    st->psl_best = st->psl;
    st->rng_ctr = (L + 63) / 64;
    st->steps = 0;
    st->near_ties = 0;
    return 0;
}

/* Neighbour autocorrelation either by the one-element flip (Sec. 3) or by the
 * definition (Eq. 2) on an explicitly flipped copy. */
static int neighbour_C(const int8_t *s, const int32_t *C, uint32_t L, uint32_t j, int mode, int8_t *tmp_s,
                       int32_t *Cn, int32_t *Cchk) {
    if (mode & ORC_MODE_FULL) {
        memcpy(tmp_s, s, L);
        tmp_s[j] = (int8_t)-tmp_s[j];
        orc_autocorr(tmp_s, L, Cn);
        return 0;
    }
    orc_flip_autocorr(s, C, L, j, Cn);
    if (mode & ORC_MODE_CROSSCHECK) {
        memcpy(tmp_s, s, L);
        tmp_s[j] = (int8_t)-tmp_s[j];
        orc_autocorr(tmp_s, L, Cchk);
        if (memcmp(Cn, Cchk, sizeof(int32_t) * L) != 0) return -2;
    }
    return 0;
}

/* Keeps the pivot if its exact F is below the lowest seen (fixed objective only). */
static void note_pivot(const orc_params *p, orc_state *st) {
    if (p->alpha1 != p->alpha2) return;
    wide_t f, b;
    memcpy(f.w, st->F, sizeof f.w);
    memcpy(b.w, st->F_best, sizeof b.w);
    if (wide_cmp(&f, &b) < 0) {
        memcpy(st->F_best, st->F, sizeof st->F_best);
        memcpy(st->fbest_seq, st->s, p->L);
    }
}

/* Runs nsteps iterations of the while loop of Alg. 1.  trace may be NULL. */
ORC_API int orc_run(const orc_params *p, orc_state *st, uint64_t nsteps, int mode, orc_trace *trace) {
    if (param_check(p)) return -1;
    const uint32_t L = p->L;
    const uint32_t N = p->n_lmt < L ? p->n_lmt : L;
    const uint32_t nflip_max = p->flip_lmt < L ? p->flip_lmt : L;
    int8_t *tmp_s = (int8_t *)malloc(L);
    int32_t *Cn = (int32_t *)malloc(sizeof(int32_t) * L);
    int32_t *Cchk = (int32_t *)malloc(sizeof(int32_t) * L);
    uint8_t *picked = (uint8_t *)calloc(L, 1);
    uint32_t *flips = (uint32_t *)malloc(sizeof(uint32_t) * (nflip_max + 1));
    int rc = 0;
    if (!tmp_s || !Cn || !Cchk || !picked || !flips) {
        rc = -1;
        goto done;
    }

    for (uint64_t t = 0; t < nsteps; t++) {
        /* start <- Rand() % L */
        uint32_t start = (uint32_t)(orc_splitmix64(p->seed, st->rng_ctr++) % L);

        /* every neighbour's |C'_k| <= |C_k| + 4, so one power table serves the window */
        wide_t *P = power_table(max_abs_sidelobe(st->C, L) + 4, st->alpha);
        if (!P) {
            rc = -1;
            goto done;
        }

        /* Neighborhood + the scan over i = 1..N (strict "<", first in scan order) */
        wide_t value_step;
        double naive_step = 0.0, naive_best = 0.0;
        uint32_t kstar = 0, naive_arg = 0;
        int32_t win_psl = 1 << 30;
        uint32_t win_psl_j = 0;
        int32_t psl_best_new = st->psl_best;
        int32_t sol_j = -1;
        for (uint32_t i = 1; i <= N; i++) {
            uint32_t j = (uint32_t)(((uint64_t)start + i) % L);
            rc = neighbour_C(st->s, st->C, L, j, mode, tmp_s, Cn, Cchk);
            if (rc) {
                free(P);
                goto done;
            }
            wide_t value_j;
            fitness_exact_tab(Cn, L, P, &value_j);
            int32_t psl_j = orc_psl(Cn, L);
            if (i == 1 || wide_cmp(&value_j, &value_step) < 0) {
                value_step = value_j;
                kstar = j;
            }
            if (psl_j < win_psl) {
                win_psl = psl_j;
                win_psl_j = j;
            }
            if (psl_j < psl_best_new) {
                psl_best_new = psl_j;
                sol_j = (int32_t)j;
            }
            if (mode & ORC_MODE_NAIVE) {
                double v = fitness_naive(Cn, L, st->alpha);
                if (i == 1 || v < naive_best) {
                    naive_best = v;
                    naive_arg = j;
                }
                if (j == kstar) naive_step = v;
            }
        }
        free(P);

        uint32_t flags = 0;
        if (sol_j >= 0) {
            memcpy(st->sol_best, st->s, L);
            st->sol_best[sol_j] = (int8_t)-st->sol_best[sol_j];
            st->psl_best = psl_best_new;
            flags |= ORC_PSL_BEST;
        }
        if ((mode & ORC_MODE_NAIVE) && naive_arg != kstar) {
            flags |= ORC_NAIVE_DIFFERS;
            st->near_ties++;
        }
        uint32_t alpha_used = st->alpha;

        /* pivot <- Flip(pivot, k) */
        orc_flip_autocorr(st->s, st->C, L, kstar, Cn);
        memcpy(st->C, Cn, sizeof(int32_t) * L);
        st->s[kstar] = (int8_t)-st->s[kstar];
        memcpy(st->F, value_step.w, sizeof st->F);
        note_pivot(p, st);

        wide_t value_local;
        memcpy(value_local.w, st->value_local, sizeof value_local.w);
        int cmp = wide_cmp(&value_step, &value_local);
        uint32_t nflip = 0;
        if (cmp < 0) {
            flags |= ORC_IMPROVED;
            st->unimproved = 0;
            memcpy(st->local_best, st->s, L);
            memcpy(st->value_local, value_step.w, sizeof st->value_local);
        } else if (cmp > 0) {
            flags |= ORC_WORSE;
            st->unimproved++;
            if (st->unimproved > p->ls_lmt) {
                /* pivot <- Rand_flip(local_best, FLIP_lmt): distinct positions */
                memset(picked, 0, L);
                while (nflip < nflip_max) {
                    uint32_t f = (uint32_t)(orc_splitmix64(p->seed, st->rng_ctr++) % L);
                    if (picked[f]) continue;
                    picked[f] = 1;
                    flips[nflip++] = f;
                }
                memcpy(st->s, st->local_best, L);
                for (uint32_t q = 0; q < nflip; q++) st->s[flips[q]] = (int8_t)-st->s[flips[q]];
                orc_autocorr(st->s, L, st->C);
                st->alpha = (st->alpha == p->alpha1) ? p->alpha2 : p->alpha1;
                uint64_t limbs[WL];
                if (orc_fitness(st->C, L, st->alpha, limbs, NULL, NULL)) {
                    rc = -1;
                    goto done;
                }
                memcpy(st->value_local, limbs, sizeof limbs);
                memcpy(st->F, limbs, sizeof limbs);
                note_pivot(p, st);
                st->unimproved = 0;
                flags |= ORC_SWITCH;
            }
        }
        st->psl = orc_psl(st->C, L);
        st->steps++;

        if (trace) {
            orc_trace *r = &trace[t];
            r->step = st->steps - 1;
            r->start = start;
            r->kstar = kstar;
            r->alpha = alpha_used;
            r->unimproved = st->unimproved;
            r->psl = st->psl;
            r->psl_best = st->psl_best;
            r->win_psl = win_psl;
            r->win_psl_j = win_psl_j;
            r->flags = flags;
            r->nflip = nflip;
            r->value_step = wide_to_double(&value_step);
            r->value_naive = naive_step;
            memcpy(r->value_exact, value_step.w, sizeof r->value_exact);
        }
    }
done:
    free(tmp_s);
    free(Cn);
    free(Cchk);
    free(picked);
    free(flips);
    return rc;
}

/* Scores one window without moving: value_j (rounded) and psl_j for i = 1..N.
 * Used to check single decisions and sampled neighbours at large L. */
ORC_API int orc_eval_neighbours(const int8_t *s, const int32_t *C, uint32_t L, uint32_t alpha, const uint32_t *js,
                                uint32_t n, uint64_t *limbs_out, int32_t *psl_out) {
    int32_t *Cn = (int32_t *)malloc(sizeof(int32_t) * L);
    wide_t *P = power_table(max_abs_sidelobe(C, L) + 4, alpha);
    if (!Cn || !P) {
        free(Cn);
        free(P);
        return -1;
    }
    for (uint32_t q = 0; q < n; q++) {
        orc_flip_autocorr(s, C, L, js[q], Cn);
        wide_t v;
        fitness_exact_tab(Cn, L, P, &v);
        if (limbs_out) memcpy(limbs_out + (size_t)q * WL, v.w, sizeof v.w);
        if (psl_out) psl_out[q] = orc_psl(Cn, L);
    }
    free(Cn);
    free(P);
    return 0;
}

ORC_API uint32_t orc_sizeof_state(void) { return (uint32_t)sizeof(orc_state); }
ORC_API uint32_t orc_sizeof_trace(void) { return (uint32_t)sizeof(orc_trace); }
ORC_API uint32_t orc_sizeof_params(void) { return (uint32_t)sizeof(orc_params); }

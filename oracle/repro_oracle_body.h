/*
 * Body of the CPU oracle, instantiated once for double and once for float by
 * repro_oracle.c (which defines the macros below before including it).
 *
 * TEST INFRASTRUCTURE ONLY -- see repro_oracle.c.
 *
 *   OT       scalar type of the state and the values (double / float)
 *   OSUF     name suffix (f64 / f32)
 *   OM       fraction bits m of OT (Sec. III-A)
 *   OW       bits between extractors W (Sec. III-C: 40 double, 18 float)
 *   OGMIN    exponent of the unit of grid index 0 (reading R3)
 *   OKMAX    largest grid index whose running sum is finite
 *   OFREXP / OLDEXP / OFABS / OFLOOR   libm functions for OT
 */

#define OCAT2(a, b) a##b
#define OCAT(a, b) OCAT2(a, b)
#define ONAME(n) OCAT(n, OCAT(_, OSUF))
#define OSTATE ONAME(orc_state)

typedef struct {
    int32_t K;      /* grid index of level 0; level l sits at grid index K - l */
    uint32_t flags; /* ORC_FLAG_* */
    OT S[ORC_LMAX]; /* running sums S^(l); 0 for levels below grid index 0 */
    int64_t C[ORC_LMAX]; /* carry-bit counts C^(l), exact integers (reading R4) */
} OSTATE;

/* ufp(x): 2^E for x = M 2^E, M in [1, 2) (Sec. III-A). */
static OT ONAME(ufp)(OT x) {
    int e;
    OFREXP(x, &e); /* x = f 2^e with f in [0.5, 1) */
    return OLDEXP((OT)1, e - 1);
}

/* ulp(x) = ufp(x) 2^-m (Sec. III-A). */
static OT ONAME(ulp)(OT x) { return OLDEXP(ONAME(ufp)(x), -OM); }

/* The empty running sum of grid index k: 1.5 ufp with ulp = 2^(g_min + k W). */
static OT ONAME(fresh)(int k) { return OLDEXP((OT)1.5, OM + OGMIN + k * OW); }

static int ONAME(present)(const OSTATE* st, int l) { return st->K - l >= 0; }

static void ONAME(init)(OSTATE* st) {
    memset(st, 0, sizeof(*st));
    st->K = 0;
    st->S[0] = ONAME(fresh)(0);
}

/* Algorithm 2, its check of the extractor's validity: drop the last level,
   demote the others, start a new first level one grid index higher. */
static void ONAME(raise)(OSTATE* st, int L) {
    OT top = st->S[0];
    for (int l = L - 1; l >= 1; --l) {
        st->S[l] = st->S[l - 1];
        st->C[l] = st->C[l - 1];
    }
    st->S[0] = (OT)1.5 * OLDEXP((OT)1, OW) * ONAME(ufp)(top);
    st->C[0] = 0;
    st->K += 1;
}

/* Keep S in [1.5, 1.75) ufp(S), moving whole quarters of ufp into C
   (Algorithm 2, carry-bit propagation). */
static void ONAME(carry)(OSTATE* st, int l) {
    OT u = ONAME(ufp)(st->S[l]);
    OT quarter = (OT)0.25 * u;
    OT d = OFLOOR((st->S[l] - (OT)1.5 * u) / quarter);
    st->S[l] = st->S[l] - d * quarter;
    st->C[l] += (int64_t)d;
}

/* One iteration of Algorithm 2 for value b. */
static void ONAME(add)(OSTATE* st, OT b, int L) {
    if (b != b) { st->flags |= ORC_FLAG_NAN; return; }
    if (OFABS(b) > OCAT(OT_MAX_, OSUF)) {
        st->flags |= (b > 0) ? ORC_FLAG_POS_INF : ORC_FLAG_NEG_INF;
        return;
    }
    /* a value that needs a level above the top grid index is flagged (R5) */
    if (OFABS(b) >= OLDEXP((OT)1, OW - 1 + OGMIN + OKMAX * OW)) {
        st->flags |= ORC_FLAG_RANGE;
        return;
    }
    /* check extractor validity, update levels if needed (threshold 2^(W-1), R1) */
    while (OFABS(b) >= OLDEXP((OT)1, OW - 1) * ONAME(ulp)(st->S[0])) ONAME(raise)(st, L);
    /* transform b level by level; the extractor is the level's constant
       1.5 ufp(S) so that ties round to even whatever S holds (R2) */
    OT r = b;
    for (int l = 0; l < L && ONAME(present)(st, l); ++l) {
        OT M = (OT)1.5 * ONAME(ufp)(st->S[l]);
        OT q = (r + M) - M;
        st->S[l] = st->S[l] + q;
        r = r - q;
    }
    /* carry-bit propagation */
    for (int l = 0; l < L && ONAME(present)(st, l); ++l) ONAME(carry)(st, l);
}

/* Move a state to the higher top grid index K (operator+=(repro) alignment,
   reading R7): levels that fall below the window are dropped. */
static void ONAME(align)(OSTATE* st, int K, int L) {
    while (st->K < K) ONAME(raise)(st, L);
}

/* operator+=(repro) (Sec. V-B); equal windows add as in eq. (2)/(3). */
static void ONAME(merge)(OSTATE* dst, const OSTATE* src_in, int L) {
    OSTATE src = *src_in;
    dst->flags |= src.flags;
    int K = dst->K > src.K ? dst->K : src.K;
    ONAME(align)(dst, K, L);
    ONAME(align)(&src, K, L);
    for (int l = 0; l < L && ONAME(present)(dst, l); ++l) {
        OT u = ONAME(ufp)(src.S[l]);
        dst->S[l] = dst->S[l] + (src.S[l] - (OT)1.5 * u);
        dst->C[l] += src.C[l];
        ONAME(carry)(dst, l);
    }
}

/* Level value (S (-) 1.5 ufp(S)) (+) 0.25 ufp(S) C of eq. (1).  Its (+) is one
   rounding of the level's exact value when both operands are exact (R4); the
   operands are formed in double, where they are exact while |T| < 2^53, and
   rounded to OT once. */
static OT ONAME(level_value)(const OSTATE* st, int l) {
    OT u = ONAME(ufp)(st->S[l]);
    double a = (double)(st->S[l] - (OT)1.5 * u);
    double c = (double)((OT)0.25 * u) * (double)st->C[l];
    return (OT)(a + c);
}

/* Finalize (eq. (1)), summed from the last level up to the first (R6). */
static OT ONAME(finalize_one)(const OSTATE* st, int L) {
    uint32_t f = st->flags;
    if ((f & (ORC_FLAG_NAN | ORC_FLAG_RANGE)) ||
        ((f & ORC_FLAG_POS_INF) && (f & ORC_FLAG_NEG_INF)))
        return (OT)NAN;
    if (f & ORC_FLAG_POS_INF) return (OT)INFINITY;
    if (f & ORC_FLAG_NEG_INF) return -(OT)INFINITY;
    int low = L - 1;
    while (!ONAME(present)(st, low)) --low;
    OT Q = ONAME(level_value)(st, low);
    for (int l = low - 1; l >= 0; --l) Q = Q + ONAME(level_value)(st, l);
    return Q;
}

/* ---------------------------------------------------------------- exports */

size_t ONAME(oracle_state_size)(void) { return sizeof(OSTATE); }

void ONAME(oracle_init)(void* states, int64_t G) {
    OSTATE* s = (OSTATE*)states;
    for (int64_t g = 0; g < G; ++g) ONAME(init)(&s[g]);
}

/* Accumulate n (key, value) rows into the G states.  Keys outside [0, G)
   are skipped; their number is returned. */
int64_t ONAME(oracle_groupby_sum)(const int32_t* keys, const OT* vals, int64_t n, int L,
                                  int64_t G, void* states) {
    OSTATE* s = (OSTATE*)states;
    int64_t bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = keys[i];
        if (k < 0 || k >= G) { ++bad; continue; }
        ONAME(add)(&s[k], vals[i], L);
    }
    return bad;
}

void ONAME(oracle_merge)(void* dst, const void* src, int L, int64_t G) {
    OSTATE* d = (OSTATE*)dst;
    const OSTATE* s = (const OSTATE*)src;
    for (int64_t g = 0; g < G; ++g) ONAME(merge)(&d[g], &s[g], L);
}

void ONAME(oracle_finalize)(const void* states, int L, int64_t G, OT* out) {
    const OSTATE* s = (const OSTATE*)states;
    for (int64_t g = 0; g < G; ++g) out[g] = ONAME(finalize_one)(&s[g], L);
}

/* Canonical integer view of a state: K, flags and the exact level integers
   T^(l) = (S - 1.5 ufp(S)) / ulp(S) + C 2^(m-2), written as hi 2^64 + lo
   with both halves signed. */
void ONAME(oracle_to_bins)(const void* states, int L, int64_t G, int32_t* K, uint32_t* flags,
                           int64_t* lo, int64_t* hi) {
    const OSTATE* s = (const OSTATE*)states;
    for (int64_t g = 0; g < G; ++g) {
        K[g] = s[g].K;
        flags[g] = s[g].flags;
        for (int l = 0; l < L; ++l) {
            __int128 t = 0;
            if (ONAME(present)(&s[g], l)) {
                OT u = ONAME(ufp)(s[g].S[l]);
                OT v = (s[g].S[l] - (OT)1.5 * u) / ONAME(ulp)(s[g].S[l]);
                t = (__int128)(int64_t)v + (__int128)s[g].C[l] * ((__int128)1 << (OM - 2));
            }
            int64_t l64 = (int64_t)(uint64_t)t; /* low 64 bits, signed */
            lo[g * L + l] = l64;
            hi[g * L + l] = (int64_t)((t - (__int128)l64) >> 64);
        }
    }
}

typedef struct {
    const int32_t* keys;
    const OT* vals;
    int64_t n, G;
    int L;
    OSTATE* states;
    int64_t bad;
} ONAME(orc_job);

static void* ONAME(orc_worker)(void* arg) {
    ONAME(orc_job)* j = (ONAME(orc_job)*)arg;
    ONAME(oracle_init)(j->states, j->G);
    j->bad = ONAME(oracle_groupby_sum)(j->keys, j->vals, j->n, j->L, j->G, j->states);
    return NULL;
}

/* Parallel over row chunks, each into a private table, then merged into
   `states` (PartitionAndAggregate with F = 1: private tables merged with
   operator+=(repro), Algorithm 4).  Returns the bad-key count, or -1 when a
   private table cannot be allocated. */
int64_t ONAME(oracle_groupby_sum_threads)(const int32_t* keys, const OT* vals, int64_t n, int L,
                                          int64_t G, void* states, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t tid[256];
    ONAME(orc_job) jobs[256];
    int64_t chunk = (n + nthreads - 1) / nthreads;
    int started = 0;
    int64_t bad = 0;
    for (int t = 0; t < nthreads; ++t) {
        int64_t a = t * chunk, b = a + chunk < n ? a + chunk : n;
        if (a >= b) break;
        jobs[t].keys = keys + a;
        jobs[t].vals = vals + a;
        jobs[t].n = b - a;
        jobs[t].G = G;
        jobs[t].L = L;
        jobs[t].bad = 0;
        jobs[t].states = (OSTATE*)malloc(sizeof(OSTATE) * (size_t)G);
        if (!jobs[t].states) { bad = -1; break; }
        if (pthread_create(&tid[t], NULL, ONAME(orc_worker), &jobs[t]) != 0) {
            free(jobs[t].states);
            bad = -1;
            break;
        }
        ++started;
    }
    for (int t = 0; t < started; ++t) {
        pthread_join(tid[t], NULL);
        if (bad >= 0) {
            ONAME(oracle_merge)(states, jobs[t].states, L, G);
            bad += jobs[t].bad;
        }
        free(jobs[t].states);
    }
    return bad;
}

#undef OSTATE
#undef ONAME
#undef OCAT
#undef OCAT2

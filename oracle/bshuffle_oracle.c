/*
 * Plain, sequential CPU oracle for the bijective shuffle of
 * "Bandwidth-Optimal Random Shuffling for GPUs" (arXiv 2106.06161).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the
 * CUDA library: only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may build, load or call it.  It shares no
 * source, header, table or constant generator with the CUDA path, and the
 * CUDA path never calls it.
 *
 * Everything here is written for obviousness, not speed: one index at a
 * time, in the order the paper states the algorithm.  The *_mt functions run
 * the same loop on several host threads over consecutive ranges of the
 * domain (a count per range, the exclusive scan of the counts in range
 * order, then a write per range from its scanned offset); they are the
 * multi-core CPU baseline and check large outputs in full, and the
 * test-suite pins them to brute force.
 *
 * Readings of the paper taken here, each with its reason:
 *   R1  mulhilo is the full 64-bit product of the 64-bit constant M0 with
 *       the zero-extended 32-bit left half, reduced mod 2^64, then split into
 *       upper and lower 32-bit words (Sec. 3.2, Listing 1 and its caption).
 *   R2  the power-of-two domain has k = max(ceil(log2 n), 4) bits: with fewer
 *       than 4 bits the left half has at most one bit, the multiply is linear
 *       over GF(2) and the cipher can only reach 2^k affine permutations
 *       (Sec. 4 takes the power of two closest above n; the 4-bit floor is
 *       the reading under which the Sec. 5 chi-squared result at n = 5 is
 *       reachable).
 *       The *_k entry points take k explicitly so the literal rule stays
 *       testable.
 *   R3  the round keys are the low 32 bits of successive SplitMix64 outputs
 *       (Steele, Lea, Flood, OOPSLA 2014) started from the 64-bit seed; the
 *       paper indexes one key per round and never gives a seed-to-key
 *       schedule.
 *   R4  an image b is kept when b < n and dropped when b >= n (Algorithm 1).
 *   R5  output convention: slot j receives X[f(i_j)], where i_j is the j-th
 *       domain index, in increasing order, whose image is kept (Algorithm 1
 *       is a gather in i-order; the exclusive scan of the keep flags is the
 *       running count used below).
 *
 * What pins the round function: the paper prints no test vector, so its
 * output bits cannot be compared with the authors' implementation.  The
 * test-suite fixes it by bijectivity (exhaustive for small k), by the
 * inversion steps of Sec. 3.2, by one round rebuilt from the prose's F/B/G
 * description, and by the round-count result of Sec. 5 (chi-squared at
 * n = 5 fails below 20 rounds and passes at 24), which the 32 x 32-bit
 * reading of "mulhilo" would not reproduce.
 */
#define _POSIX_C_SOURCE 200809L  /* sysconf, pthreads */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* Philox multiplier named in Listing 1 (Sec. 3.2), from Salmon et al. */
static const uint64_t ORACLE_M0 = 0xD2B74407B1CE6E93ULL;
/* Reading R2: smallest domain exponent. */
static const uint32_t ORACLE_K_MIN = 4;
/* SplitMix64 increment (golden-ratio gamma), Steele-Lea-Flood 2014. */
static const uint64_t ORACLE_SPLITMIX_GAMMA = 0x9E3779B97F4A7C15ULL;

/* ------------------------------------------------------------------ */
/* Domain (Sec. 4, first paragraph; reading R2)                        */
/* ------------------------------------------------------------------ */

/* Smallest k with 2^k >= n, never below ORACLE_K_MIN.  n = 0 gives 0. */
uint32_t oracle_domain_bits(uint64_t n)
{
    uint32_t k = 0;
    if (n == 0)
        return 0;
    while (k < 64 && ((uint64_t)1 << k) < n)
        k++;
    if (k < ORACLE_K_MIN)
        k = ORACLE_K_MIN;
    return k;
}

/* ------------------------------------------------------------------ */
/* Round keys (reading R3)                                             */
/* ------------------------------------------------------------------ */

static uint64_t oracle_splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state += ORACLE_SPLITMIX_GAMMA;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void oracle_round_keys(uint64_t seed, uint32_t rounds, uint32_t *keys)
{
    uint64_t state = seed;
    uint32_t r;
    for (r = 0; r < rounds; r++)
        keys[r] = (uint32_t)oracle_splitmix64_next(&state);
}

/* ------------------------------------------------------------------ */
/* VariablePhilox bijection on [0, 2^k) (Sec. 3.2, Listing 1)          */
/* ------------------------------------------------------------------ */

static uint64_t oracle_mask(uint32_t bits)
{
    return bits >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << bits) - 1);
}

/*
 * Forward cipher.  The k-bit value is split into a left half of floor(k/2)
 * bits (state[0]) and a right half of ceil(k/2) bits (state[1]); each round
 *   - multiplies M0 by the left half (64-bit product, reading R1),
 *   - forms the new right half from the low product word shifted up by the
 *     odd-bit count (R - L) with the top bit of the old right half moved in
 *     underneath (the function G of Sec. 3.2 mixing the odd bit b),
 *   - forms the new left half as (high product word) XOR key XOR (old right
 *     half), masked to L bits (L' = F_k(L) xor R in Sec. 3.2),
 * and the halves are joined back as left << R | right.
 */
uint64_t oracle_varphilox(uint64_t x, uint32_t k, const uint32_t *keys, uint32_t rounds)
{
    const uint32_t left_bits = k / 2;
    const uint32_t right_bits = k - left_bits;
    const uint64_t left_mask = oracle_mask(left_bits);
    const uint64_t right_mask = oracle_mask(right_bits);
    uint32_t state0 = (uint32_t)(x >> right_bits);
    uint32_t state1 = (uint32_t)(x & right_mask);
    uint32_t r;

    for (r = 0; r < rounds; r++) {
        uint64_t product = ORACLE_M0 * (uint64_t)state0;  /* mod 2^64 */
        uint32_t hi = (uint32_t)(product >> 32);
        uint32_t lo = (uint32_t)product;
        lo = (uint32_t)(lo << (right_bits - left_bits)) | (uint32_t)(state1 >> left_bits);
        state0 = (uint32_t)(((uint64_t)(hi ^ keys[r]) ^ state1) & left_mask);
        state1 = (uint32_t)((uint64_t)lo & right_mask);
    }
    return ((uint64_t)state0 << right_bits) | (uint64_t)state1;
}

/* Multiplicative inverse of an odd a modulo 2^64 by Newton's iteration
 * x <- x (2 - a x); a*a = 1 mod 8 gives 3 correct bits to start, and each
 * step doubles them (3, 6, 12, 24, 48, 96). */
static uint64_t oracle_inverse_mod_2_64(uint64_t a)
{
    uint64_t x = a;
    int it;
    for (it = 0; it < 5; it++)
        x = x * (2 - a * x);
    return x;
}

uint64_t oracle_m0_inverse(void)
{
    return oracle_inverse_mod_2_64(ORACLE_M0);
}

/*
 * Inverse cipher, the inversion steps of Sec. 3.2 applied round by round in
 * reverse key order:
 *   (B_k(L), b) = G^-1(R', b')   -- the low bit of the new right half is the
 *                                   old top bit b (odd k only); the bits
 *                                   above it are the low L bits of M0 * L,
 *   L = B_k^-1(B_k(L))           -- multiply by M0^-1 modulo 2^L,
 *   R = F_k(L) xor L'            -- recompute the high product word.
 */
uint64_t oracle_varphilox_inverse(uint64_t y, uint32_t k, const uint32_t *keys, uint32_t rounds)
{
    const uint32_t left_bits = k / 2;
    const uint32_t right_bits = k - left_bits;
    const uint32_t odd = right_bits - left_bits;          /* 0 or 1 */
    const uint64_t left_mask = oracle_mask(left_bits);
    const uint64_t right_mask = oracle_mask(right_bits);
    const uint64_t m0_inv = oracle_inverse_mod_2_64(ORACLE_M0);
    uint64_t new_left = y >> right_bits;
    uint64_t new_right = y & right_mask;
    uint32_t r;

    for (r = rounds; r-- > 0;) {
        uint64_t b = odd ? (new_right & 1) : 0;
        uint64_t b_of_left = odd ? (new_right >> 1) : new_right;   /* = M0*L mod 2^L */
        uint64_t left = (b_of_left * m0_inv) & left_mask;
        uint64_t product = ORACLE_M0 * left;
        uint64_t hi = product >> 32;
        uint64_t right_low = (new_left ^ hi ^ (uint64_t)keys[r]) & left_mask;
        uint64_t right = right_low | (b << left_bits);
        new_left = left;
        new_right = right;
    }
    return (new_left << right_bits) | new_right;
}

void oracle_varphilox_array(const uint64_t *x, uint64_t *y, uint64_t count, uint32_t k,
                            const uint32_t *keys, uint32_t rounds)
{
    uint64_t t;
    for (t = 0; t < count; t++)
        y[t] = oracle_varphilox(x[t], k, keys, rounds);
}

void oracle_varphilox_inverse_array(const uint64_t *y, uint64_t *x, uint64_t count, uint32_t k,
                                    const uint32_t *keys, uint32_t rounds)
{
    uint64_t t;
    for (t = 0; t < count; t++)
        x[t] = oracle_varphilox_inverse(y[t], k, keys, rounds);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (Sec. 4): evaluate, flag, exclusive scan, gather         */
/* ------------------------------------------------------------------ */

/*
 * idx[j] = f(i_j) for the j-th kept domain index, i ascending over [0, 2^k).
 * The running count `j` is the exclusive scan of the keep flags.  Returns the
 * number of kept indices (n for a bijection on a domain with 2^k >= n).
 */
uint64_t oracle_indices_k(uint64_t *idx, uint64_t n, uint32_t k, uint64_t seed, uint32_t rounds)
{
    uint32_t keys[256];
    uint64_t domain, i, j = 0;
    if (n == 0 || rounds > 256 || k > 40)
        return 0;
    oracle_round_keys(seed, rounds, keys);
    domain = (uint64_t)1 << k;
    for (i = 0; i < domain; i++) {
        uint64_t b = oracle_varphilox(i, k, keys, rounds);
        int flag = (b < n) ? 1 : 0;
        if (flag) {
            if (j < n)
                idx[j] = b;
            j++;
        }
    }
    return j;
}

uint64_t oracle_indices(uint64_t *idx, uint64_t n, uint64_t seed, uint32_t rounds)
{
    return oracle_indices_k(idx, n, oracle_domain_bits(n), seed, rounds);
}

/* Y[out_idx] = X[b] (Algorithm 1), elements of elem_bytes bytes.  Returns the
 * number of elements written. */
uint64_t oracle_permute_k(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint32_t k,
                          uint64_t seed, uint32_t rounds)
{
    const unsigned char *x = (const unsigned char *)in;
    unsigned char *y = (unsigned char *)out;
    uint32_t keys[256];
    uint64_t domain, i, out_idx = 0;
    if (n == 0 || rounds > 256 || k > 40)
        return 0;
    oracle_round_keys(seed, rounds, keys);
    domain = (uint64_t)1 << k;
    for (i = 0; i < domain; i++) {
        uint64_t b = oracle_varphilox(i, k, keys, rounds);
        if (b < n) {
            memcpy(y + out_idx * elem_bytes, x + b * elem_bytes, elem_bytes);
            out_idx++;
        }
    }
    return out_idx;
}

uint64_t oracle_permute(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                        uint32_t rounds)
{
    return oracle_permute_k(in, out, n, elem_bytes, oracle_domain_bits(n), seed, rounds);
}

/* The first `slots` output elements of oracle_permute (the same loop, stopped
 * once `slots` elements have been written): a bounded sample of a large
 * shuffle for CPU timing. */
uint64_t oracle_permute_first(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                              uint32_t rounds, uint64_t slots)
{
    const unsigned char *x = (const unsigned char *)in;
    unsigned char *y = (unsigned char *)out;
    uint32_t keys[256];
    uint32_t k = oracle_domain_bits(n);
    uint64_t domain, i, out_idx = 0;
    if (n == 0 || rounds > 256 || k > 40)
        return 0;
    oracle_round_keys(seed, rounds, keys);
    domain = (uint64_t)1 << k;
    for (i = 0; i < domain && out_idx < slots; i++) {
        uint64_t b = oracle_varphilox(i, k, keys, rounds);
        if (b < n) {
            memcpy(y + out_idx * elem_bytes, x + b * elem_bytes, elem_bytes);
            out_idx++;
        }
    }
    return out_idx;
}

/* The inverse shuffle: out[f(i_j)] = in[j], so that inverse(permute(x)) = x. */
uint64_t oracle_inverse(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                        uint32_t rounds)
{
    const unsigned char *x = (const unsigned char *)in;
    unsigned char *y = (unsigned char *)out;
    uint32_t keys[256];
    uint32_t k = oracle_domain_bits(n);
    uint64_t domain, i, j = 0;
    if (n == 0 || rounds > 256 || k > 40)
        return 0;
    oracle_round_keys(seed, rounds, keys);
    domain = (uint64_t)1 << k;
    for (i = 0; i < domain; i++) {
        uint64_t b = oracle_varphilox(i, k, keys, rounds);
        if (b < n) {
            memcpy(y + b * elem_bytes, x + j * elem_bytes, elem_bytes);
            j++;
        }
    }
    return j;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 over domain ranges: count, exclusive scan, then write     */
/* ------------------------------------------------------------------ */

/*
 * Number of domain indices i in [i0, i1) whose image f(i) is kept (below n),
 * on the domain of n.  Summed over a partition of [0, 2^k) into consecutive
 * ranges, these counts scanned in range order give each range's first output
 * slot: Algorithm 1's exclusive scan taken at the range boundaries.
 */
uint64_t oracle_count_range(uint64_t n, uint64_t seed, uint32_t rounds, uint64_t i0, uint64_t i1)
{
    uint32_t keys[256];
    uint32_t k = oracle_domain_bits(n);
    uint64_t domain, i, count = 0;
    if (n == 0 || rounds > 256 || k > 40)
        return 0;
    oracle_round_keys(seed, rounds, keys);
    domain = (uint64_t)1 << k;
    if (i1 > domain)
        i1 = domain;
    for (i = i0; i < i1; i++)
        if (oracle_varphilox(i, k, keys, rounds) < n)
            count++;
    return count;
}

/*
 * The same Algorithm 1 run by T host threads, each over one of T consecutive
 * ranges of the domain: every thread counts its kept indices, the counts are
 * scanned in range order (exclusive), and every thread then writes its kept
 * images (or elements) from its scanned offset.  The output equals the
 * sequential oracle_indices_k / oracle_permute_k; this is the multi-core
 * count-then-gather form of the method, used as a CPU baseline and to check
 * large GPU outputs in full.
 */
typedef struct {
    uint64_t lo, hi;            /* domain range [lo, hi) */
    uint64_t n;
    uint32_t k, rounds;
    const uint32_t *keys;
    uint64_t count;             /* kept indices in the range (pass 1) */
    uint64_t offset;            /* first output slot of the range (pass 2) */
    uint64_t *idx;              /* indices output, or NULL */
    const unsigned char *in;    /* permute input, or NULL */
    unsigned char *out;         /* permute output */
    uint32_t elem_bytes;
} oracle_range_job;

static void *oracle_range_count(void *arg)
{
    oracle_range_job *job = (oracle_range_job *)arg;
    uint64_t i, count = 0;
    for (i = job->lo; i < job->hi; i++)
        if (oracle_varphilox(i, job->k, job->keys, job->rounds) < job->n)
            count++;
    job->count = count;
    return NULL;
}

static void *oracle_range_write(void *arg)
{
    oracle_range_job *job = (oracle_range_job *)arg;
    uint64_t i, j = job->offset;
    for (i = job->lo; i < job->hi; i++) {
        uint64_t b = oracle_varphilox(i, job->k, job->keys, job->rounds);
        if (b < job->n) {
            if (job->idx != NULL)
                job->idx[j] = b;
            else
                memcpy(job->out + j * job->elem_bytes, job->in + b * job->elem_bytes, job->elem_bytes);
            j++;
        }
    }
    return NULL;
}

/* Runs fn over every job, one thread each (the calling thread takes job 0). */
static int oracle_run_jobs(void *(*fn)(void *), oracle_range_job *jobs, uint32_t threads)
{
    pthread_t tid[256];
    uint32_t t, started = 0;
    int rc = 0;
    for (t = 1; t < threads; t++) {
        if (pthread_create(&tid[t], NULL, fn, &jobs[t]) != 0) {
            rc = -1;
            break;
        }
        started = t;
    }
    if (rc == 0)
        fn(&jobs[0]);
    for (t = 1; t <= started; t++)
        pthread_join(tid[t], NULL);
    return rc;
}

uint32_t oracle_default_threads(void)
{
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1)
        return 1;
    return c > 256 ? 256u : (uint32_t)c;
}

/* Count, scan, write: the threaded form of Algorithm 1 (idx or in/out). */
static uint64_t oracle_algorithm1_mt(uint64_t *idx, const void *in, void *out, uint64_t n, uint32_t elem_bytes,
                                     uint32_t k, uint64_t seed, uint32_t rounds, uint32_t threads)
{
    oracle_range_job jobs[256];
    uint32_t keys[256];
    uint64_t domain, total = 0;
    uint32_t t;
    if (n == 0 || rounds > 256 || k > 40)
        return 0;
    if (threads == 0)
        threads = oracle_default_threads();
    if (threads > 256)
        threads = 256;
    oracle_round_keys(seed, rounds, keys);
    domain = (uint64_t)1 << k;
    if (threads > domain)
        threads = (uint32_t)domain;
    for (t = 0; t < threads; t++) {
        memset(&jobs[t], 0, sizeof(jobs[t]));
        jobs[t].lo = domain / threads * t;
        jobs[t].hi = t + 1 == threads ? domain : domain / threads * (t + 1);
        jobs[t].n = n;
        jobs[t].k = k;
        jobs[t].rounds = rounds;
        jobs[t].keys = keys;
        jobs[t].idx = idx;
        jobs[t].in = (const unsigned char *)in;
        jobs[t].out = (unsigned char *)out;
        jobs[t].elem_bytes = elem_bytes;
    }
    if (oracle_run_jobs(oracle_range_count, jobs, threads) != 0)
        return 0;
    for (t = 0; t < threads; t++) {   /* exclusive scan of the range counts */
        jobs[t].offset = total;
        total += jobs[t].count;
    }
    if (total != n)
        return total;                 /* not a bijection onto [0, n): write nothing */
    if (oracle_run_jobs(oracle_range_write, jobs, threads) != 0)
        return 0;
    return total;
}

/* The kept elements of the domain range [first, end) in increasing domain
 * order (the output slots of that range, from the range's first slot), on
 * `threads` host threads over sub-ranges: a bounded sample of a large
 * shuffle for CPU timing.  Returns the number written. */
uint64_t oracle_permute_range_mt(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                                 uint32_t rounds, uint64_t first, uint64_t end, uint32_t threads)
{
    oracle_range_job jobs[256];
    uint32_t keys[256];
    uint32_t k = oracle_domain_bits(n);
    uint64_t total = 0, span;
    uint32_t t;
    if (in == NULL || out == NULL || elem_bytes == 0 || n == 0 || rounds > 256 || k > 40)
        return 0;
    if (end > ((uint64_t)1 << k))
        end = (uint64_t)1 << k;
    if (first >= end)
        return 0;
    if (threads == 0)
        threads = oracle_default_threads();
    if (threads > 256)
        threads = 256;
    span = end - first;
    if (threads > span)
        threads = (uint32_t)span;
    oracle_round_keys(seed, rounds, keys);
    for (t = 0; t < threads; t++) {
        memset(&jobs[t], 0, sizeof(jobs[t]));
        jobs[t].lo = first + span / threads * t;
        jobs[t].hi = t + 1 == threads ? end : first + span / threads * (t + 1);
        jobs[t].n = n;
        jobs[t].k = k;
        jobs[t].rounds = rounds;
        jobs[t].keys = keys;
        jobs[t].in = (const unsigned char *)in;
        jobs[t].out = (unsigned char *)out;
        jobs[t].elem_bytes = elem_bytes;
    }
    if (oracle_run_jobs(oracle_range_count, jobs, threads) != 0)
        return 0;
    for (t = 0; t < threads; t++) {
        jobs[t].offset = total;
        total += jobs[t].count;
    }
    if (oracle_run_jobs(oracle_range_write, jobs, threads) != 0)
        return 0;
    return total;
}

uint64_t oracle_indices_mt(uint64_t *idx, uint64_t n, uint64_t seed, uint32_t rounds, uint32_t threads)
{
    return oracle_algorithm1_mt(idx, NULL, NULL, n, 0, oracle_domain_bits(n), seed, rounds, threads);
}

uint64_t oracle_permute_mt(const void *in, void *out, uint64_t n, uint32_t elem_bytes, uint64_t seed,
                           uint32_t rounds, uint32_t threads)
{
    if (in == NULL || out == NULL || elem_bytes == 0)
        return 0;
    return oracle_algorithm1_mt(NULL, in, out, n, elem_bytes, oracle_domain_bits(n), seed, rounds, threads);
}

/* count permutations of length n (as idx arrays, uint32) from seeds
 * seed0, seed0+1, ...; used by the statistical tests of Sec. 5. */
void oracle_sample_permutations(uint32_t *perms, uint32_t n, uint64_t seed0, uint64_t count,
                                uint32_t rounds)
{
    uint64_t s, j;
    uint64_t *idx = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    for (s = 0; s < count; s++) {
        oracle_indices(idx, n, seed0 + s, rounds);
        for (j = 0; j < n; j++)
            perms[s * n + j] = (uint32_t)idx[j];
    }
    free(idx);
}

/* ------------------------------------------------------------------ */
/* LCG bijection (Sec. 3.1, Eq. lcg) on the same padded domain         */
/* ------------------------------------------------------------------ */

/*
 * y = (a x + c) mod 2^k with a odd, so a is coprime to 2^k and x -> y is a
 * bijection of [0, 2^k).  Reading R6: the paper gives no seed-to-(a, c)
 * mapping; here a = (first SplitMix64 output of the seed) with its low bit
 * set, c = the second output, both reduced mod 2^k.
 */
void oracle_lcg_params(uint64_t seed, uint32_t k, uint64_t *a, uint64_t *c)
{
    uint64_t state = seed;
    uint64_t mask = oracle_mask(k);
    *a = (oracle_splitmix64_next(&state) | 1) & mask;
    *c = oracle_splitmix64_next(&state) & mask;
}

uint64_t oracle_lcg(uint64_t x, uint32_t k, uint64_t a, uint64_t c)
{
    return (a * x + c) & oracle_mask(k);
}

/* Algorithm 1 with the LCG as f: idx[j] = f(i_j). */
uint64_t oracle_indices_lcg(uint64_t *idx, uint64_t n, uint64_t seed)
{
    uint32_t k = oracle_domain_bits(n);
    uint64_t a, c, domain, i, j = 0;
    if (n == 0 || k > 40)
        return 0;
    oracle_lcg_params(seed, k, &a, &c);
    domain = (uint64_t)1 << k;
    for (i = 0; i < domain; i++) {
        uint64_t b = oracle_lcg(i, k, a, c);
        if (b < n) {
            if (j < n)
                idx[j] = b;
            j++;
        }
    }
    return j;
}

/* count LCG permutations of length n from seeds seed0, seed0+1, ... */
void oracle_sample_permutations_lcg(uint32_t *perms, uint32_t n, uint64_t seed0, uint64_t count)
{
    uint64_t s, j;
    uint64_t *idx = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    for (s = 0; s < count; s++) {
        oracle_indices_lcg(idx, n, seed0 + s);
        for (j = 0; j < n; j++)
            perms[s * n + j] = (uint32_t)idx[j];
    }
    free(idx);
}

/* ------------------------------------------------------------------ */
/* Fisher-Yates (Sec. 1): the sequential baseline, timing only          */
/* ------------------------------------------------------------------ */

/* Durstenfeld's in-place form; bounded integers by rejection from a
 * SplitMix64 stream (no modulo bias). */
void oracle_fisher_yates(void *data, uint64_t n, uint32_t elem_bytes, uint64_t seed)
{
    unsigned char *a = (unsigned char *)data;
    unsigned char tmp[256];
    uint64_t state = seed, i;
    if (n < 2 || elem_bytes > sizeof(tmp))
        return;
    for (i = n - 1; i > 0; i--) {
        uint64_t bound = i + 1;
        uint64_t limit = ~(uint64_t)0 - (~(uint64_t)0 % bound);
        uint64_t r, j;
        do {
            r = oracle_splitmix64_next(&state);
        } while (r >= limit);
        j = r % bound;
        memcpy(tmp, a + i * elem_bytes, elem_bytes);
        memcpy(a + i * elem_bytes, a + j * elem_bytes, elem_bytes);
        memcpy(a + j * elem_bytes, tmp, elem_bytes);
    }
}

/* ------------------------------------------------------------------ */
/* Permutation Monte Carlo test statistic (application named in Sec. 1) */
/* ------------------------------------------------------------------ */

/*
 * For each b < count: shuffle x (length n) with seed base_seed + b and
 * return T_b = mean(y[0:n1]) - mean(y[n1:n]), summed in FP64 in slot order.
 */
void oracle_mc_statistics(const float *x, uint64_t n, uint64_t n1, uint64_t base_seed,
                          uint64_t count, uint32_t rounds, double *T)
{
    uint32_t keys[256];
    uint32_t k = oracle_domain_bits(n);
    uint64_t domain = (uint64_t)1 << k;
    uint64_t b, i;
    if (n == 0 || n1 == 0 || n1 >= n || rounds > 256)
        return;
    for (b = 0; b < count; b++) {
        double sum1 = 0.0, sum2 = 0.0;
        uint64_t slot = 0;
        oracle_round_keys(base_seed + b, rounds, keys);
        for (i = 0; i < domain; i++) {
            uint64_t src = oracle_varphilox(i, k, keys, rounds);
            if (src < n) {
                if (slot < n1)
                    sum1 += (double)x[src];
                else
                    sum2 += (double)x[src];
                slot++;
            }
        }
        T[b] = sum1 / (double)n1 - sum2 / (double)(n - n1);
    }
}

/* ------------------------------------------------------------------ */
/* Kendall discordant-pair count for the Mallows kernel (Sec. 5)        */
/* ------------------------------------------------------------------ */

static uint64_t oracle_merge_count(uint32_t *a, uint32_t *tmp, uint32_t lo, uint32_t hi)
{
    uint32_t mid, i, j, t;
    uint64_t inv;
    if (hi - lo < 2)
        return 0;
    mid = lo + (hi - lo) / 2;
    inv = oracle_merge_count(a, tmp, lo, mid) + oracle_merge_count(a, tmp, mid, hi);
    i = lo;
    j = mid;
    t = lo;
    while (i < mid && j < hi) {
        if (a[i] <= a[j]) {
            tmp[t++] = a[i++];
        } else {
            inv += mid - i;
            tmp[t++] = a[j++];
        }
    }
    while (i < mid)
        tmp[t++] = a[i++];
    while (j < hi)
        tmp[t++] = a[j++];
    memcpy(a + lo, tmp + lo, sizeof(uint32_t) * (hi - lo));
    return inv;
}

/*
 * n_dis(s, t) = #{i < j : (s(i) < s(j)) != (t(i) < t(j))} for permutations s,
 * t of [0, n) in one-line notation: order the positions by s and count the
 * inversions of t read in that order (merge sort, Knight 1966).
 */
uint64_t oracle_kendall_discordant(const uint32_t *s, const uint32_t *t, uint32_t n)
{
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *seq = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t i;
    uint64_t inv;
    for (i = 0; i < n; i++)
        order[s[i]] = i;              /* order[r] = position holding rank r in s */
    for (i = 0; i < n; i++)
        seq[i] = t[order[i]];
    inv = oracle_merge_count(seq, tmp, 0, n);
    free(order);
    free(seq);
    free(tmp);
    return inv;
}

/* Pairwise counts for consecutive pairs (perms[2p], perms[2p+1]), the pairing
 * of the unbiased MMD estimate in Sec. 5. */
void oracle_kendall_pairs(const uint32_t *perms, uint32_t n, uint64_t num_pairs, uint64_t *out)
{
    uint64_t p;
    for (p = 0; p < num_pairs; p++)
        out[p] = oracle_kendall_discordant(perms + (2 * p) * n, perms + (2 * p + 1) * n, n);
}

/* ------------------------------------------------------------------ */
/* Shapley values by permutation sampling (application named in Sec. 1) */
/* ------------------------------------------------------------------ */

/*
 * Weighted voting game v(S) = 1 if sum_{i in S} w_i >= quota, else 0.  The
 * Shapley value of player i is the probability, over uniform orders of the
 * players, that i is pivotal: the running weight of the players before i is
 * below the quota and adding w_i reaches it.  Sample s orders the players by
 * the shuffle of Algorithm 1 with seed seed0 + s (slot j holds player
 * f(i_j)); counts[i] = number of samples in which player i is pivotal.
 * With quota 0 or above the total weight no player is ever pivotal.
 */
void oracle_shapley_voting(const uint32_t *w, uint64_t n, uint64_t quota, uint64_t seed0,
                           uint64_t samples, uint32_t rounds, uint64_t *counts)
{
    uint32_t keys[256];
    uint32_t k;
    uint64_t domain, s, i;
    memset(counts, 0, sizeof(uint64_t) * n);
    if (n == 0 || quota == 0 || rounds > 256)
        return;
    k = oracle_domain_bits(n);
    domain = (uint64_t)1 << k;
    for (s = 0; s < samples; s++) {
        uint64_t before = 0;
        oracle_round_keys(seed0 + s, rounds, keys);
        for (i = 0; i < domain; i++) {
            uint64_t player = oracle_varphilox(i, k, keys, rounds);
            if (player >= n)
                continue;
            if (before < quota && before + w[player] >= quota) {
                counts[player]++;
                break;
            }
            before += w[player];
        }
    }
}

/*
 * shaken_oracle.c -- plain, slow, single-threaded CPU oracle for the shaken
 * dynamics (D'Autilia, Andrianaivo, Troiani, "Parallel simulation of
 * two-dimensional Ising models using Probabilistic Cellular Automata").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header or table with the
 * CUDA path: the Philox generator, the threshold table and the field
 * computation are all written here a second time, on purpose.
 *
 * What it computes, step by step in the paper's notation:
 *   - the lattice Lambda = (Z/LZ)^2, site x = (i, j), linear index u = j*L + i;
 *     neighbours x^up = (i, j+1), x^right = (i+1, j), x^down = (i, j-1),
 *     x^left = (i-1, j)                                   (Section 2, "The model")
 *   - left field  <-h_x(sigma) = J(sigma_{x down} + sigma_{x left}) + q sigma_x
 *     right field ->h_x(tau)   = J(tau_{x up}     + tau_{x right})  + q tau_x
 *                                                           (Eq. "urdl")
 *   - half-step A (odd times, Eq. "leftTrans"): every tau_u is redrawn
 *     independently with P(tau_u = +1 | sigma) = e^{h} / (2 cosh h),
 *     h = <-h_u(sigma);
 *   - half-step B (even times, Eq. "rightTrans"): every sigma_u is redrawn with
 *     P(sigma_u = +1 | tau) = e^{h} / (2 cosh h), h = ->h_u(tau);
 *   - one full step = A then B (Algorithm 3, with the half-step order of the
 *     equations, see the readings below);
 *   - magnetisation m = |Lambda|^-1 sum sigma_x (Section 3.1) and the pair
 *     Hamiltonian H(sigma, tau) = -sum_x [J sigma_x (tau_{x up} + tau_{x right})
 *     + q sigma_x tau_x] (Eq. "gs_ham2"), kept as exact integer sums.
 *
 * Readings where the paper leaves a choice open (each fixed here and in the
 * library, identically):
 *   R1  half-step order: A (left field, writes tau) then B (right field,
 *       writes sigma), as in Eqs. leftTrans/rightTrans and the Hamiltonian's
 *       geometry; Algorithm 3 lists the two collect calls in the mirror order.
 *   R2  sign: P(+1) = e^{h}/(2 cosh h) = 1/(1 + e^{-2h}) (ferromagnetic).
 *   R3  the uniform draw is a 32-bit integer r and the comparison is r < T(h)
 *       with an integer threshold T(h) (below), so P(+1) = T(h) / 2^32.
 *   R4  threshold rounding: for h > 0, T = min(2^32 - 1, floor(2^32 p(h)))
 *       with p evaluated in IEEE double; for h < 0, T(h) = 2^32 - T(-h);
 *       T(0) = 2^31.
 *   R5  random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 *       random numbers: as easy as 1, 2, 3", SC 2011) keyed by the 64-bit seed.
 *       Sites are grouped in blocks of 32 consecutive linear indices
 *       (block w = u >> 5, position p = u & 31).  For half-step index
 *       hs (2t for A of step t, 2t+1 for B) the block draws eight Philox
 *       blocks, call c = 0..7, with counter (hs, w, lattice_id, c) and key
 *       (seed_lo, seed_hi); call c yields the four words R[4c..4c+3].  The
 *       32-bit uniform of site u is the p-th column of that 32x32 bit matrix,
 *       most significant bit first:  r(u) = sum_b bit_p(R[b]) * 2^(31-b).
 *       Every site thus receives exactly one 32-bit Philox-derived uniform.
 *   R6  random initial state: the same construction with counter
 *       (plane, w, lattice_id, 256 + c) and the init seed; spin up iff
 *       r(u) < 2^31.
 *   R7  observables of step t are taken on the pair (sigma_t, tau_t) at the
 *       end of the step: M_sigma, M_tau, S_q = sum sigma_x tau_x,
 *       S_J = sum sigma_x (tau_{x up} + tau_{x right}),
 *       C_nn = sum sigma_x (sigma_{x up} + sigma_{x right}).
 *
 * Spins are int8 values +1 / -1 stored row-major, plane[u] with u = j*L + i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 constants as published by Salmon et al. (2011): the two round
 * multipliers and the two Weyl key increments. */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

/* One Philox4x32 round: two 32x32->64 products, the high halves xored with
 * the other two counter words and the round key, the words permuted. */
static void orc_philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

/* Philox4x32-10: ten rounds, the key bumped by the Weyl constants between
 * rounds (round r uses key + r*W). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += ORC_PHILOX_W0;
            k[1] += ORC_PHILOX_W1;
        }
        orc_philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* The 32 uniforms of block w (reading R5 / R6): fills r[0..31] with the
 * site uniforms r(32w + p), p = 0..31. */
void orc_block_uniforms(uint64_t seed, uint32_t c0, uint32_t w, uint32_t lattice_id,
                        uint32_t domain, uint32_t r[32]) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t R[32];
    for (uint32_t c = 0; c < 8; ++c) {
        uint32_t ctr[4] = {c0, w, lattice_id, domain * 256u + c};
        orc_philox4x32_10(ctr, key, &R[4 * c]);
    }
    for (int p = 0; p < 32; ++p) {
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) {
            uint32_t bit = (R[b] >> p) & 1u;
            v |= bit << (31 - b);
        }
        r[p] = v;
    }
}

/* ------------------------------------------------------------ thresholds */

/* T(h) of reading R4 for one field value h. */
static uint32_t orc_threshold_of(double h) {
    if (h == 0.0) return 0x80000000u;
    double a = fabs(h);
    double p = 1.0 / (1.0 + exp(-2.0 * a));         /* e^a / (2 cosh a) */
    double scaled = ldexp(p, 32);
    double fl = floor(scaled);
    uint32_t t_pos = (fl >= 4294967295.0) ? 0xffffffffu : (uint32_t)fl;
    if (h > 0.0) return t_pos;
    return (uint32_t)(0u - t_pos);                  /* 2^32 - T(-h) */
}

/* The six thresholds, indexed k = 3*[s = +1] + n, where s is the spin at the
 * site itself and n in {0,1,2} is the number of +1 among its two neighbours
 * in the field; the field is h = q*s + J*(2n - 2).  Returns 0, or -1 when q
 * or J is not finite. */
int orc_thresholds(double q, double J, uint32_t T[6]) {
    if (!isfinite(q) || !isfinite(J)) return -1;
    for (int s01 = 0; s01 < 2; ++s01) {
        double s = s01 ? 1.0 : -1.0;
        for (int n = 0; n < 3; ++n) {
            double h = q * s + J * (double)(2 * n - 2);
            T[3 * s01 + n] = orc_threshold_of(h);
        }
    }
    return 0;
}

/* ------------------------------------------------------------- lattice */

static int64_t orc_wrap(int64_t a, int64_t L) {
    int64_t m = a % L;
    return m < 0 ? m + L : m;
}

/* Initial state of one plane (reading R6).  kind: 0 all up, 1 all down,
 * 2 random with p = 1/2. */
void orc_init(int8_t* plane, int L, int kind, uint64_t init_seed,
              uint32_t lattice_id, uint32_t plane_index) {
    int64_t N = (int64_t)L * L;
    if (kind == 0 || kind == 1) {
        for (int64_t u = 0; u < N; ++u) plane[u] = (kind == 0) ? 1 : -1;
        return;
    }
    uint32_t r[32];
    for (int64_t u = 0; u < N; ++u) {
        if ((u & 31) == 0 || u == 0)
            orc_block_uniforms(init_seed, plane_index, (uint32_t)(u >> 5), lattice_id, 1u, r);
        plane[u] = (r[u & 31] < 0x80000000u) ? 1 : -1;
    }
}

/* One half-step restricted to the rows [row0, row1) of the output plane.
 * half = 0: half-step A, dst = tau drawn from src = sigma with the left field.
 * half = 1: half-step B, dst = sigma drawn from src = tau with the right field.
 * hs is the half-step index (2t or 2t+1).  Sites are visited in increasing
 * linear order. */
void orc_halfstep_rows(int half, const int8_t* src, int8_t* dst, int L,
                       const uint32_t T[6], uint64_t seed, uint32_t lattice_id,
                       uint32_t hs, int row0, int row1) {
    uint32_t r[32];
    int64_t cached_w = -1;
    for (int64_t j = row0; j < row1; ++j) {
        for (int64_t i = 0; i < L; ++i) {
            int64_t u = j * L + i;
            int64_t n1, n2;
            if (half == 0) {            /* x^down and x^left */
                n1 = orc_wrap(j - 1, L) * L + i;
                n2 = j * L + orc_wrap(i - 1, L);
            } else {                    /* x^up and x^right */
                n1 = orc_wrap(j + 1, L) * L + i;
                n2 = j * L + orc_wrap(i + 1, L);
            }
            int s_up = src[u] > 0;
            int n_up = (src[n1] > 0) + (src[n2] > 0);
            uint32_t thr = T[3 * s_up + n_up];
            int64_t w = u >> 5;
            if (w != cached_w) {
                orc_block_uniforms(seed, hs, (uint32_t)w, lattice_id, 0u, r);
                cached_w = w;
            }
            dst[u] = (r[u & 31] < thr) ? 1 : -1;
        }
    }
}

/* The five exact integer sums of reading R7 for the pair (sigma, tau). */
void orc_observables(const int8_t* sigma, const int8_t* tau, int L, int64_t out[5]) {
    int64_t m_s = 0, m_t = 0, s_q = 0, s_j = 0, c_nn = 0;
    for (int64_t j = 0; j < L; ++j) {
        for (int64_t i = 0; i < L; ++i) {
            int64_t u = j * L + i;
            int64_t up = orc_wrap(j + 1, L) * L + i;
            int64_t rt = j * L + orc_wrap(i + 1, L);
            m_s += sigma[u];
            m_t += tau[u];
            s_q += (int64_t)sigma[u] * tau[u];
            s_j += (int64_t)sigma[u] * (tau[up] + tau[rt]);
            c_nn += (int64_t)sigma[u] * (sigma[up] + sigma[rt]);
        }
    }
    out[0] = m_s; out[1] = m_t; out[2] = s_q; out[3] = s_j; out[4] = c_nn;
}

/* n full steps t = t0 .. t0+n-1 of the alternate dynamics, in place on
 * (sigma, tau).  obs (nullable) receives n rows of the five sums. */
int orc_run(int8_t* sigma, int8_t* tau, int L, double q, double J, uint64_t seed,
            uint32_t lattice_id, uint64_t t0, uint64_t n, int64_t* obs) {
    uint32_t T[6];
    if (L < 2 || orc_thresholds(q, J, T) != 0) return -1;
    if (t0 + n > 0x80000000ull) return -1;
    for (uint64_t s = 0; s < n; ++s) {
        uint64_t t = t0 + s;
        orc_halfstep_rows(0, sigma, tau, L, T, seed, lattice_id, (uint32_t)(2 * t), 0, L);
        orc_halfstep_rows(1, tau, sigma, L, T, seed, lattice_id, (uint32_t)(2 * t + 1), 0, L);
        if (obs) orc_observables(sigma, tau, L, obs + 5 * s);
    }
    return 0;
}

/* M independent chains on one small torus: chain m uses lattice id
 * id0 + m, starts from the state given by init_sigma (N values) and runs n
 * steps.  The final sigma of chain m is written as an integer code: bit u set
 * iff sigma_u = +1 (requires N <= 63).  Used by the statistical tests. */
int orc_many_chains(int L, double q, double J, uint64_t seed, uint32_t id0, int64_t M,
                    const int8_t* init_sigma, uint64_t n, uint64_t* codes_sigma,
                    uint64_t* codes_tau) {
    int64_t N = (int64_t)L * L;
    if (N > 63) return -1;
    int8_t* s = (int8_t*)malloc((size_t)N);
    int8_t* t = (int8_t*)malloc((size_t)N);
    if (!s || !t) { free(s); free(t); return -1; }
    for (int64_t m = 0; m < M; ++m) {
        memcpy(s, init_sigma, (size_t)N);
        memset(t, 1, (size_t)N);
        if (orc_run(s, t, L, q, J, seed, id0 + (uint32_t)m, 0, n, NULL) != 0) {
            free(s); free(t); return -1;
        }
        uint64_t cs = 0, ct = 0;
        for (int64_t u = 0; u < N; ++u) {
            if (s[u] > 0) cs |= 1ull << u;
            if (t[u] > 0) ct |= 1ull << u;
        }
        codes_sigma[m] = cs;
        if (codes_tau) codes_tau[m] = ct;
    }
    free(s); free(t);
    return 0;
}

/* Diagonal spin-spin sums of Section 3.3 (Table 1), translation-averaged:
 * out[k] = sum_x s_x s_{x+(l,l)} (SW-NE), out[n+k] = sum_x s_x s_{x+(l,-l)}
 * (NW-SE: the pair (0,l), (l,0)), x = (i, j), l = lags[k]. */
void orc_diag_correlations(const int8_t* s, int L, const int* lags, int n, int64_t* out) {
    for (int k = 0; k < n; ++k) {
        int64_t l = lags[k], a = 0, b = 0;
        for (int64_t j = 0; j < L; ++j) {
            for (int64_t i = 0; i < L; ++i) {
                int64_t x = j * L + i;
                int64_t y1 = orc_wrap(j + l, L) * L + orc_wrap(i + l, L);
                int64_t y2 = orc_wrap(j - l, L) * L + orc_wrap(i + l, L);
                a += (int64_t)s[x] * s[y1];
                b += (int64_t)s[x] * s[y2];
            }
        }
        out[k] = a;
        out[n + k] = b;
    }
}

/* ------------------------------------------------- checkerboard heat bath */

/* The comparison dynamics of Section 3.2 for the square-lattice Ising model
 * H_G(s) = -J sum_x s_x (s_{x up} + s_{x right}): the even sites (i + j even)
 * are redrawn given the odd ones, then the odd sites given the even ones,
 * each with P(s_x = +1) = e^{h}/(2 cosh h), h = J (sum of the four
 * neighbours) (heat bath).  Thresholds by the rule of reading R4, indexed by
 * the number n = 0..4 of + neighbours, h = J (2n - 4).  The uniforms are
 * spent only on the sites being redrawn: those sites, numbered row by row,
 * a = j (L/2) + floor(i/2) (each row holds one of every pair of columns
 * (2m, 2m+1)), take the block uniforms of reading R5 with counter
 * (hs, a >> 5, lattice_id, 512 + c), column a & 31. */
int orc_checkerboard_thresholds(double J, uint32_t T[5]) {
    if (!isfinite(J)) return -1;
    for (int n = 0; n < 5; ++n) T[n] = orc_threshold_of(J * (double)(2 * n - 4));
    return 0;
}

void orc_checkerboard_halfstep(int8_t* s, int L, const uint32_t T[5], uint64_t seed,
                               uint32_t lattice_id, uint32_t hs, int parity) {
    uint32_t r[32];
    int64_t cached_w = -1;
    for (int64_t j = 0; j < L; ++j) {
        for (int64_t i = 0; i < L; ++i) {
            if (((i + j) & 1) != parity) continue;
            int64_t u = j * L + i;
            int n = (s[orc_wrap(j + 1, L) * L + i] > 0) + (s[orc_wrap(j - 1, L) * L + i] > 0) +
                    (s[j * L + orc_wrap(i + 1, L)] > 0) + (s[j * L + orc_wrap(i - 1, L)] > 0);
            int64_t a = j * (L / 2) + i / 2;   /* index among the redrawn sites */
            int64_t w = a >> 5;
            if (w != cached_w) {
                orc_block_uniforms(seed, hs, (uint32_t)w, lattice_id, 2u, r);
                cached_w = w;
            }
            s[u] = (r[a & 31] < T[n]) ? 1 : -1;
        }
    }
}

/* n full steps t = t0 .. t0+n-1 (even sites with hs = 2t, then odd sites with
 * hs = 2t + 1), in place; obs (nullable) receives n rows of (M, C_nn) where
 * C_nn = sum_x s_x (s_{x up} + s_{x right}), so H_G = -J C_nn.  L even. */
int orc_checkerboard_run(int8_t* s, int L, double J, uint64_t seed, uint32_t lattice_id,
                         uint64_t t0, uint64_t n, int64_t* obs) {
    uint32_t T[5];
    if (L < 2 || (L & 1) || orc_checkerboard_thresholds(J, T) != 0) return -1;
    if (t0 + n > 0x80000000ull) return -1;
    for (uint64_t k = 0; k < n; ++k) {
        uint64_t t = t0 + k;
        orc_checkerboard_halfstep(s, L, T, seed, lattice_id, (uint32_t)(2 * t), 0);
        orc_checkerboard_halfstep(s, L, T, seed, lattice_id, (uint32_t)(2 * t + 1), 1);
        if (obs) {
            int64_t m = 0, c = 0;
            for (int64_t j = 0; j < L; ++j)
                for (int64_t i = 0; i < L; ++i) {
                    int64_t u = j * L + i;
                    m += s[u];
                    c += (int64_t)s[u] * (s[orc_wrap(j + 1, L) * L + i] + s[j * L + orc_wrap(i + 1, L)]);
                }
            obs[2 * k] = m;
            obs[2 * k + 1] = c;
        }
    }
    return 0;
}

/* ---- coupling from the past (Propp-Wilson, Section 3.2) -------------------
 *
 * Both dynamics are monotone for J, q >= 0 (the order sigma >= eta of the
 * paper's footnote is kept by every step driven by the same uniforms), so it
 * is enough to follow the chains started from all + and all -.  Time runs
 * from -2^k to 0.  The randomness of the step from time -s to -s + 1 (s >= 1)
 * must not depend on k: it is that of forward step index s - 1 (half-steps
 * 2(s-1) and 2(s-1) + 1).  Attempt k = 0, 1, 2, ... runs both chains from
 * time -2^k to 0; the first attempt after which they agree returns their
 * common state at time 0, a draw from the stationary law.  For the shaken
 * dynamics the state compared and returned is sigma (tau is overwritten by
 * the first half-step and carries no state).
 * dyn 0 = shaken (q, J), dyn 1 = checkerboard heat bath (J; L even).
 * Returns the k of the successful attempt, or -1 when none up to k_max
 * coalesced (sample then holds nothing), -2 on bad arguments. */
int orc_cftp(int dyn, int L, double q, double J, uint64_t seed, uint32_t lattice_id, int k_max,
             int8_t* sample) {
    if (L < 2 || k_max < 0 || k_max > 30 || (dyn != 0 && dyn != 1)) return -2;
    if (dyn == 1 && (L & 1)) return -2;
    uint32_t T6[6], T5[5];
    if (dyn == 0 && orc_thresholds(q, J, T6) != 0) return -2;
    if (dyn == 1 && orc_checkerboard_thresholds(J, T5) != 0) return -2;
    const int64_t N = (int64_t)L * L;
    int8_t* top = (int8_t*)malloc((size_t)N);
    int8_t* bot = (int8_t*)malloc((size_t)N);
    int8_t* ttop = (int8_t*)malloc((size_t)N);
    int8_t* tbot = (int8_t*)malloc((size_t)N);
    int result = -1;
    for (int k = 0; k <= k_max && result < 0; ++k) {
        for (int64_t u = 0; u < N; ++u) {
            top[u] = 1;
            bot[u] = -1;
            ttop[u] = tbot[u] = 1;
        }
        for (int64_t s = (int64_t)1 << k; s >= 1; --s) {
            const uint64_t t = (uint64_t)(s - 1);
            if (dyn == 0) {
                orc_run(top, ttop, L, q, J, seed, lattice_id, t, 1, NULL);
                orc_run(bot, tbot, L, q, J, seed, lattice_id, t, 1, NULL);
            } else {
                orc_checkerboard_run(top, L, J, seed, lattice_id, t, 1, NULL);
                orc_checkerboard_run(bot, L, J, seed, lattice_id, t, 1, NULL);
            }
        }
        if (memcmp(top, bot, (size_t)N) == 0) {
            memcpy(sample, top, (size_t)N);
            result = k;
        }
    }
    free(top);
    free(bot);
    free(ttop);
    free(tbot);
    return result;
}

/* M independent perfect samples (lattice ids id0 .. id0 + M - 1) as state
 * codes (bit u set iff the spin at u is +1; N <= 64) and their k. */
int orc_cftp_many(int dyn, int L, double q, double J, uint64_t seed, uint32_t id0, int64_t M, int k_max,
                  uint64_t* codes, int32_t* ks) {
    const int64_t N = (int64_t)L * L;
    if (N > 64 || M < 0) return -2;
    int8_t* s = (int8_t*)malloc((size_t)N);
    for (int64_t m = 0; m < M; ++m) {
        const int k = orc_cftp(dyn, L, q, J, seed, id0 + (uint32_t)m, k_max, s);
        if (k == -2) {
            free(s);
            return -2;
        }
        ks[m] = k;
        uint64_t c = 0;
        if (k >= 0)
            for (int64_t u = 0; u < N; ++u)
                if (s[u] > 0) c |= (uint64_t)1 << u;
        codes[m] = c;
    }
    free(s);
    return 0;
}

/*
 * fcs_oracle.c -- plain, slow, FP64 CPU oracle for Fast Count Sketch (FCS).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant generator with the CUDA library; it is an independent restatement
 * of "Efficient Tensor Contraction via Fast Count Sketch" (Cao & Liu).
 *
 * Every routine follows the plain definition it cites, in the paper's order,
 * with no blocking, fusion or reordering.  Arithmetic is FP64; inputs arrive
 * as FP64 arrays that hold values already rounded to FP32 by the caller.
 * Indices are 0-based throughout: the paper's 1-based bin
 * h_1(i_1)+...+h_N(i_N)-N+1 becomes h_1(i_1)+...+h_N(i_N) here.
 *
 * Hash family (the paper only asks for "2-wise independent" pairs, Def. 1
 * and Def. 4): Carter-Wegman multiply-mod-prime over p = 2^61-1,
 *     h(i) = ((a_h*i + b_h) mod p) mod J,
 *     s(i) = 1 - 2*(((a_s*i + b_s) mod p) & 1),
 * with (a_h, b_h, a_s, b_s) drawn from the SplitMix64 generator (Steele, Lea
 * & Flood, OOPSLA 2014) seeded with `seed`, four draws per (d, n) in the order
 * d = 0..D-1, n = 0..N-1:  a = 1 + x mod (p-1),  b = x mod p.
 * The k-th SplitMix64 output (k = 0, 1, ...) is mix(seed + (k+1)*gamma).
 *
 * Parity status per routine is recorded in the test suite's pins; every
 * routine here has at least one pin (closed form, library routine, invariant
 * or brute force) except where its header comment says "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static const uint64_t P61 = 0x1FFFFFFFFFFFFFFFULL; /* 2^61 - 1 */

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood 2014): k-th output of the stream seeded   */
/* with `seed`.  Counter-based: the state after k+1 steps is seed+(k+1)*g.   */
/* ------------------------------------------------------------------------ */
uint64_t fcso_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Coefficients (a_h, b_h, a_s, b_s) for every (d, n): out[(d*N+n)*4 + 0..3]. */
void fcso_hash_coeffs(uint64_t seed, int N, int D, uint64_t *out)
{
    uint64_t k = 0;
    for (int d = 0; d < D; ++d)
        for (int n = 0; n < N; ++n) {
            uint64_t *c = out + ((size_t)d * N + n) * 4;
            c[0] = 1 + fcso_splitmix64(seed, k++) % (P61 - 1);
            c[1] = fcso_splitmix64(seed, k++) % P61;
            c[2] = 1 + fcso_splitmix64(seed, k++) % (P61 - 1);
            c[3] = fcso_splitmix64(seed, k++) % P61;
        }
}

/* Hash tables for D independent sketches of an order-N tensor (Def. 4).
 * h, s are laid out [D][sum_n I_n]; mode n starts at offset sum_{m<n} I_m.  */
void fcso_make_hashes(uint64_t seed, int N, const int64_t *I, const int32_t *J,
                      int D, int32_t *h, int8_t *s)
{
    int64_t total = 0;
    for (int n = 0; n < N; ++n) total += I[n];
    uint64_t *coef = (uint64_t *)malloc(sizeof(uint64_t) * 4 * (size_t)N * D);
    fcso_hash_coeffs(seed, N, D, coef);
    for (int d = 0; d < D; ++d) {
        int64_t off = 0;
        for (int n = 0; n < N; ++n) {
            const uint64_t *c = coef + ((size_t)d * N + n) * 4;
            for (int64_t i = 0; i < I[n]; ++i) {
                uint64_t vh = (uint64_t)(((u128)c[0] * (uint64_t)i + c[1]) % P61);
                uint64_t vs = (uint64_t)(((u128)c[2] * (uint64_t)i + c[3]) % P61);
                h[(size_t)d * total + off + i] = (int32_t)(vh % (uint64_t)J[n]);
                s[(size_t)d * total + off + i] = (int8_t)(1 - 2 * (int)(vs & 1));
            }
            off += I[n];
        }
    }
    free(coef);
}

/* ------------------------------------------------------------------------ */
/* Count Sketch of a vector, Def. 1:  CS(x)_j = sum_{h(i)=j} s(i) x(i).      */
/* ------------------------------------------------------------------------ */
void fcso_count_sketch(int64_t I, const double *x, const int32_t *h,
                       const int8_t *s, int64_t J, double *out)
{
    for (int64_t j = 0; j < J; ++j) out[j] = 0.0;
    for (int64_t i = 0; i < I; ++i) out[h[i]] += (double)s[i] * x[i];
}

/* ------------------------------------------------------------------------ */
/* Full linear convolution (the circled-asterisk of eq. FCS_syn):            */
/*   out[k] = sum_{i+j=k} a[i] b[j],  length la+lb-1.                        */
/* Each output is an independent sum over i in increasing order.             */
/* ------------------------------------------------------------------------ */
void fcso_linear_convolve(int64_t la, const double *a, int64_t lb,
                          const double *b, double *out)
{
    int64_t lo = la + lb - 1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < lo; ++k) {
        int64_t i0 = k - (lb - 1) > 0 ? k - (lb - 1) : 0;
        int64_t i1 = k < la - 1 ? k : la - 1;
        double acc = 0.0;
        for (int64_t i = i0; i <= i1; ++i) acc += a[i] * b[k - i];
        out[k] = acc;
    }
}

static int64_t jtilde(int N, const int32_t *J)
{
    int64_t t = 1;
    for (int n = 0; n < N; ++n) t += (int64_t)J[n] - 1;
    return t;
}

/* ------------------------------------------------------------------------ */
/* FCS of a general (dense) tensor, eq. FCS_asyn:                            */
/*   FCS(T)_j = sum_{H(i_1..i_N)=j} S(i_1..i_N) T(i_1..i_N),                 */
/*   H = sum_n h_n(i_n),  S = prod_n s_n(i_n).                               */
/* T is addressed through element strides (any layout); every multi-index   */
/* is visited once in lexicographic order.  h, s: [D][sum I] as above.       */
/* out: [D][Jt], Jt = sum J_n - N + 1.                                       */
/* ------------------------------------------------------------------------ */
void fcso_fcs_dense(int N, const int64_t *I, const int64_t *stride,
                    const int32_t *J, int D, const double *T, const int32_t *h,
                    const int8_t *s, double *out)
{
    int64_t Jt = jtilde(N, J), total = 0, numel = 1;
    int64_t off[16];
    for (int n = 0; n < N; ++n) { off[n] = total; total += I[n]; numel *= I[n]; }
#pragma omp parallel for schedule(static)
    for (int d = 0; d < D; ++d) {
        const int32_t *hd = h + (size_t)d * total;
        const int8_t *sd = s + (size_t)d * total;
        double *o = out + (size_t)d * Jt;
        for (int64_t j = 0; j < Jt; ++j) o[j] = 0.0;
        int64_t idx[16];
        for (int n = 0; n < N; ++n) idx[n] = 0;
        for (int64_t e = 0; e < numel; ++e) {
            int64_t bin = 0, addr = 0;
            double sign = 1.0;
            for (int n = 0; n < N; ++n) {
                bin += hd[off[n] + idx[n]];
                sign *= (double)sd[off[n] + idx[n]];
                addr += idx[n] * stride[n];
            }
            o[bin] += sign * T[addr];
            for (int n = N - 1; n >= 0; --n) {   /* next multi-index */
                if (++idx[n] < I[n]) break;
                idx[n] = 0;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Tensor Sketch, Def. 2 (every hash length J):                              */
/*   TS(T)_j = sum_{H(i_1..i_N)=j} S(i_1..i_N) T(i_1..i_N),                  */
/*   H = (sum_n h_n(i_n)) mod J (0-based form of the paper's                 */
/*   (h_1 + ... + h_N - N) mod J + 1),  S = prod_n s_n(i_n).                 */
/* Same traversal and table layout as fcso_fcs_dense; out: [D][J].           */
/* ------------------------------------------------------------------------ */
void fcso_ts_dense(int N, const int64_t *I, const int64_t *stride, int32_t J, int D,
                   const double *T, const int32_t *h, const int8_t *s, double *out)
{
    int64_t total = 0, numel = 1;
    int64_t off[16];
    for (int n = 0; n < N; ++n) { off[n] = total; total += I[n]; numel *= I[n]; }
#pragma omp parallel for schedule(static)
    for (int d = 0; d < D; ++d) {
        const int32_t *hd = h + (size_t)d * total;
        const int8_t *sd = s + (size_t)d * total;
        double *o = out + (size_t)d * J;
        for (int64_t j = 0; j < J; ++j) o[j] = 0.0;
        int64_t idx[16];
        for (int n = 0; n < N; ++n) idx[n] = 0;
        for (int64_t e = 0; e < numel; ++e) {
            int64_t sum = 0, addr = 0;
            double sign = 1.0;
            for (int n = 0; n < N; ++n) {
                sum += hd[off[n] + idx[n]];
                sign *= (double)sd[off[n] + idx[n]];
                addr += idx[n] * stride[n];
            }
            o[sum % J] += sign * T[addr];
            for (int n = N - 1; n >= 0; --n) {
                if (++idx[n] < I[n]) break;
                idx[n] = 0;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Long hash pair of Def. 4 for one sketch: for the column-major linear      */
/* index l = sum_n i_n prod_{m<n} I_m (0-based form of the paper's formula), */
/*   H(l) = sum_n h_n(i_n),  S(l) = prod_n s_n(i_n).                         */
/* hd, sd point at one sketch's tables ([sum I]).  H, S have prod I entries. */
/* ------------------------------------------------------------------------ */
void fcso_long_hash(int N, const int64_t *I, const int32_t *hd,
                    const int8_t *sd, int32_t *H, int8_t *S)
{
    int64_t numel = 1, off[16], total = 0;
    for (int n = 0; n < N; ++n) { off[n] = total; total += I[n]; numel *= I[n]; }
    for (int64_t l = 0; l < numel; ++l) {
        int64_t rem = l, bin = 0;
        int sign = 1;
        for (int n = 0; n < N; ++n) {          /* i_1 varies fastest */
            int64_t in = rem % I[n];
            rem /= I[n];
            bin += hd[off[n] + in];
            sign *= sd[off[n] + in];
        }
        H[l] = (int32_t)bin;
        S[l] = (int8_t)sign;
    }
}

/* ------------------------------------------------------------------------ */
/* Materialise a CP tensor T = sum_r lambda_r u_r^(1) o ... o u_r^(N)        */
/* (the CPD of the notation section) in C order.  U[n] is I_n x R row-major  */
/* with leading dimension ldU[n].  lambda may be NULL (all ones).            */
/* ------------------------------------------------------------------------ */
void fcso_cp_to_dense(int N, const int64_t *I, int64_t R,
                      const double *const *U, const int64_t *ldU,
                      const double *lambda, double *T)
{
    int64_t numel = 1;
    for (int n = 0; n < N; ++n) numel *= I[n];
    int64_t idx[16];
    for (int n = 0; n < N; ++n) idx[n] = 0;
    for (int64_t e = 0; e < numel; ++e) {
        double acc = 0.0;
        for (int64_t r = 0; r < R; ++r) {
            double prod = lambda ? lambda[r] : 1.0;
            for (int n = 0; n < N; ++n) prod *= U[n][idx[n] * ldU[n] + r];
            acc += prod;
        }
        T[e] = acc;
        for (int n = N - 1; n >= 0; --n) {
            if (++idx[n] < I[n]) break;
            idx[n] = 0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* FCS of a CP tensor, eq. FCS_syn, second line:                             */
/*   FCS(T) = sum_r lambda_r CS_1(u_r^(1)) (*) ... (*) CS_N(u_r^(N)),        */
/* with (*) the full linear convolution computed directly (no FFT).          */
/* out: [D][Jt].                                                             */
/* ------------------------------------------------------------------------ */
void fcso_fcs_cp(int N, const int64_t *I, const int32_t *J, int64_t R, int D,
                 const double *const *U, const int64_t *ldU,
                 const double *lambda, const int32_t *h, const int8_t *s,
                 double *out)
{
    int64_t Jt = jtilde(N, J), total = 0, off[16], Imax = 0;
    for (int n = 0; n < N; ++n) {
        off[n] = total; total += I[n];
        if (I[n] > Imax) Imax = I[n];
    }
    double *col = (double *)malloc(sizeof(double) * (size_t)Imax);
    double *cs = (double *)malloc(sizeof(double) * (size_t)Jt);
    double *acc = (double *)malloc(sizeof(double) * (size_t)Jt);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)Jt);
    for (int d = 0; d < D; ++d) {
        double *o = out + (size_t)d * Jt;
        for (int64_t j = 0; j < Jt; ++j) o[j] = 0.0;
        for (int64_t r = 0; r < R; ++r) {
            int64_t len = 0;
            for (int n = 0; n < N; ++n) {
                for (int64_t i = 0; i < I[n]; ++i) col[i] = U[n][i * ldU[n] + r];
                fcso_count_sketch(I[n], col, h + (size_t)d * total + off[n],
                                  s + (size_t)d * total + off[n], J[n], cs);
                if (n == 0) {
                    for (int64_t j = 0; j < J[0]; ++j) acc[j] = cs[j];
                    len = J[0];
                } else {
                    fcso_linear_convolve(len, acc, J[n], cs, tmp);
                    len = len + J[n] - 1;
                    for (int64_t j = 0; j < len; ++j) acc[j] = tmp[j];
                }
            }
            double lr = lambda ? lambda[r] : 1.0;
            for (int64_t j = 0; j < Jt; ++j) o[j] += lr * acc[j];
        }
    }
    free(col); free(cs); free(acc); free(tmp);
}

/* Sketch of the rank-1 tensor v_1 o ... o v_N for sketch d, skipping mode   */
/* `skip` (-1 = none), as the chained convolution of the per-mode CS.        */
/* Writes `*len` entries into w (capacity Jt).                               */
static void rank1_sketch(int N, const int64_t *I, const int32_t *J,
                         const int64_t *off, int64_t total, int d,
                         const double *const *v, const int32_t *h,
                         const int8_t *s, int skip, double *w, int64_t *len,
                         double *cs, double *tmp)
{
    int64_t L = 0;
    for (int n = 0; n < N; ++n) {
        if (n == skip) continue;
        fcso_count_sketch(I[n], v[n], h + (size_t)d * total + off[n],
                          s + (size_t)d * total + off[n], J[n], cs);
        if (L == 0) {
            for (int64_t j = 0; j < J[n]; ++j) w[j] = cs[j];
            L = J[n];
        } else {
            fcso_linear_convolve(L, w, J[n], cs, tmp);
            L = L + J[n] - 1;
            for (int64_t j = 0; j < L; ++j) w[j] = tmp[j];
        }
    }
    if (L == 0) { w[0] = 1.0; L = 1; }   /* N == 1 with the only mode free */
    *len = L;
}

/* ------------------------------------------------------------------------ */
/* T(v_1,...,v_N) estimate, eq. T_uvw first line, for each sketch d:         */
/*   e_d = < FCS_d(T), FCS_d(v_1 o ... o v_N) >,                             */
/* where FCS_d of the rank-1 tensor is the chained linear convolution of     */
/* the per-mode CS (eq. FCS_syn with R = 1).  fcsT: [D][Jt], v[n]: I_n.      */
/* out: [D].                                                                 */
/* ------------------------------------------------------------------------ */
void fcso_contract_all(int N, const int64_t *I, const int32_t *J, int D,
                       const double *fcsT, const double *const *v,
                       const int32_t *h, const int8_t *s, double *out)
{
    int64_t Jt = jtilde(N, J), total = 0, off[16];
    for (int n = 0; n < N; ++n) { off[n] = total; total += I[n]; }
    double *w = (double *)malloc(sizeof(double) * (size_t)Jt);
    double *cs = (double *)malloc(sizeof(double) * (size_t)Jt);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)Jt);
    for (int d = 0; d < D; ++d) {
        int64_t L;
        rank1_sketch(N, I, J, off, total, d, v, h, s, -1, w, &L, cs, tmp);
        double acc = 0.0;
        for (int64_t j = 0; j < Jt; ++j) acc += fcsT[(size_t)d * Jt + j] * w[j];
        out[d] = acc;
    }
    free(w); free(cs); free(tmp);
}

/* ------------------------------------------------------------------------ */
/* T(.., I, ..) estimate with free mode m, eq. T_Ivw first line (and the     */
/* ALS columns, which free any mode):                                        */
/*   est_d[i] = < FCS_d(T), FCS_d(v_1 o .. e_i (mode m) .. o v_N) >.         */
/* The rank-1 sketch with e_i in mode m is s_m(i) times the convolution w of */
/* the other modes' CS shifted by h_m(i), so                                 */
/*   est_d[i] = s_m(i) * sum_k FCS_d(T)[h_m(i) + k] * w[k].                  */
/* v[m] is ignored.  out: [D][I_m].                                          */
/* ------------------------------------------------------------------------ */
void fcso_contract_free(int N, const int64_t *I, const int32_t *J, int D,
                        int m, const double *fcsT, const double *const *v,
                        const int32_t *h, const int8_t *s, double *out)
{
    int64_t Jt = jtilde(N, J), total = 0, off[16];
    for (int n = 0; n < N; ++n) { off[n] = total; total += I[n]; }
    double *w = (double *)malloc(sizeof(double) * (size_t)Jt);
    double *cs = (double *)malloc(sizeof(double) * (size_t)Jt);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)Jt);
    for (int d = 0; d < D; ++d) {
        int64_t L;
        rank1_sketch(N, I, J, off, total, d, v, h, s, m, w, &L, cs, tmp);
        const int32_t *hm = h + (size_t)d * total + off[m];
        const int8_t *sm = s + (size_t)d * total + off[m];
        const double *x = fcsT + (size_t)d * Jt;
        for (int64_t i = 0; i < I[m]; ++i) {
            double acc = 0.0;
            for (int64_t k = 0; k < L; ++k) acc += x[hm[i] + k] * w[k];
            out[(size_t)d * I[m] + i] = (double)sm[i] * acc;
        }
    }
    free(w); free(cs); free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Median of D independent estimates (Sec. 4 opening): sort; odd D takes the */
/* middle value, even D the mean of the two middle values.                   */
/* vals: [D][count] -> out: [count] (elementwise over the second axis).      */
/* ------------------------------------------------------------------------ */
void fcso_median(int D, int64_t count, const double *vals, double *out)
{
    double *buf = (double *)malloc(sizeof(double) * (size_t)D);
    for (int64_t c = 0; c < count; ++c) {
        for (int d = 0; d < D; ++d) buf[d] = vals[(size_t)d * count + c];
        for (int a = 1; a < D; ++a) {        /* insertion sort */
            double key = buf[a];
            int b = a - 1;
            while (b >= 0 && buf[b] > key) { buf[b + 1] = buf[b]; --b; }
            buf[b + 1] = key;
        }
        out[c] = (D % 2) ? buf[D / 2] : 0.5 * (buf[D / 2 - 1] + buf[D / 2]);
    }
    free(buf);
}

/* ------------------------------------------------------------------------ */
/* Entry recovery (the decompressing rules of the Kronecker and contraction  */
/* compression subsections), for each sketch d and sample q:                 */
/*   raw_d[q] = prod_n s_n(i_n) * sketch_d[ sum_n h_n(i_n) ],                */
/* (the printed mod(., 4J-3) never wraps and is dropped); out = median_d.    */
/* idx: [M][N] int32 multi-indices.  raw: [D][M] (may be NULL).  out: [M].   */
/* ------------------------------------------------------------------------ */
void fcso_recover(int N, const int64_t *I, const int32_t *J, int D,
                  const double *sketch, const int32_t *h, const int8_t *s,
                  int64_t M, const int32_t *idx, double *raw, double *out)
{
    int64_t Jt = jtilde(N, J), total = 0, off[16];
    for (int n = 0; n < N; ++n) { off[n] = total; total += I[n]; }
    double *r = raw ? raw : (double *)malloc(sizeof(double) * (size_t)D * M);
    for (int d = 0; d < D; ++d)
        for (int64_t q = 0; q < M; ++q) {
            int64_t bin = 0;
            double sign = 1.0;
            for (int n = 0; n < N; ++n) {
                int64_t in = idx[q * N + n];
                bin += h[(size_t)d * total + off[n] + in];
                sign *= (double)s[(size_t)d * total + off[n] + in];
            }
            r[(size_t)d * M + q] = sign * sketch[(size_t)d * Jt + bin];
        }
    fcso_median(D, M, r, out);
    if (!raw) free(r);
}

/* ------------------------------------------------------------------------ */
/* Sketch of an outer product from the sketches of its factors (the FCS of   */
/* a Kronecker product): FCS(A o B) = FCS(A) (*) FCS(B), the full linear     */
/* convolution (what the zero-padded FFT product of that subsection          */
/* computes).  fa: [D][La], fb: [D][Lb] -> out: [D][La+Lb-1].                */
/* ------------------------------------------------------------------------ */
void fcso_outer_combine(int D, int64_t La, const double *fa, int64_t Lb,
                        const double *fb, double *out)
{
    for (int d = 0; d < D; ++d)
        fcso_linear_convolve(La, fa + (size_t)d * La, Lb, fb + (size_t)d * Lb,
                             out + (size_t)d * (La + Lb - 1));
}

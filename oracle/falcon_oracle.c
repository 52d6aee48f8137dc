/*
 * falcon_oracle.c -- plain, slow CPU oracle of the Falcon codec
 * (Falcon: GPU-Based Floating-point Adaptive Lossless Compression, arXiv 2511.04140).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls this
 * file; only the test-suite, the smoke check and the CPU-baseline leg of the bench do.
 * It shares no code, header, table or constant generator with the CUDA library: the
 * powers of ten come from the C library's correctly rounded decimal parser (strtod /
 * strtof), the arithmetic is plain IEEE FP64/FP32 compiled with -ffp-contract=off.
 *
 * Every function follows one passage of the paper, in the paper's order and notation:
 *   - Def. 1/2, Eq. 2 (Sec. 2.2)            decimal place alpha, decimal significand beta
 *   - Alg. 2 (Sec. 3.2.2), Thm 4            DPAndDSCalculation
 *   - Sec. 3.2.3, Eq. 4, Thm 5              digit transformation (Case 1 / Case 2)
 *   - Eq. 5                                 delta + zigzag
 *   - Sec. 3.3, Fig. 8                      adaptive sparse/dense bit-plane encoding,
 *                                           chunk record layout
 *   - Sec. 3.4, Alg. 3                      size array + concatenated chunk records
 *   - Sec. 4                                decompression = exact inverse
 *
 * Readings where the paper is silent (numbered as in the design notes):
 *   R1  -0.0, NaN (any payload), +-inf and subnormals are exceptions (alpha,beta)=(23,16)
 *       (FP32: (11,8)); they force the chunk to Case 2 (bit-exact through BinLong).
 *   R3  floor(log10|v|) := the largest k with |v| >= fl(10^k) (fl = correctly rounded).
 *   R4  the product v (x) 10^alpha is the IEEE multiply, no contraction.
 *   R5  round() is half-away-from-zero (ties cannot occur where it matters).
 *   R6  a Case-1 chunk is additionally checked value by value: g_i / 10^alpha_max must
 *       reproduce v_i bit for bit, otherwise the chunk falls back to Case 2.
 *   R7  integer arithmetic is modulo 2^64 (2^32 for FP32); zigzag uses an arithmetic
 *       shift; z_1 is stored raw, little-endian, 8 bytes (FP32: 4).
 *   R8  row 1 of the transposed matrix is the most significant plane (bit w-1).
 *   R9  bits are MSB-first everywhere: column 8j+i -> bit 7-i of row byte j; bitmap bit
 *       for row byte j -> bit 7-(j%8) of bitmap byte j/8; the flag bits of rows 1..w are
 *       the last w bits of ceil(w/8) bytes read MSB-first; 0 = sparse, 1 = dense.
 *   R10 sparse iff lambda > cols/64; a tie is stored dense.
 *   R11 a chunk of m values has cols = round_up(m-1, 64) columns; missing columns are
 *       zero pads that count in bytes, bitmap and lambda but not in w. m = 1 -> w = 0.
 *   R12 a Case-2 record stores the sentinels (alpha,beta_hat) = (23,16) (FP32: (11,8));
 *       a decoder treats a record as Case 1 iff alpha <= 22 and beta_hat <= 15
 *       (FP32: alpha <= 10, beta_hat <= 7).
 *   R13 the u32 size array precedes the records.
 *   R14 FP32: alpha <= 10, beta <= 7, mu = |x| * 2^-23, x = v * 10^alpha computed exactly
 *       (in FP64), round trip and decode are fl32((float)g / (float)10^alpha).
 *   R16 block sizes: 2 <= B <= 1025 (Sec. 3.3's n = 64k + 1 with the implementation's
 *       n = 1025 as the largest chunk).
 *   R18 FP16 (half precision; Sec. 2.1 says the method extends to other precisions and
 *       fixes nothing more): alpha <= 4 (10^4 is the largest power of ten exact in binary16),
 *       beta <= 3 (10^3 < 2^11 <= 10^4), mu = |x| * 2^-10 (the 11-bit significand's unit, as
 *       2^-52 and 2^-23 are for FP64 and FP32), x = v * 10^alpha exact (in FP64); the round
 *       trip and the decode are fl16(g / 10^alpha), correctly rounded (ties to even); the
 *       Case-2 sentinels are (5, 4); zigzag and deltas are modulo 2^16; z_1 takes 2 bytes and
 *       w <= 16.  -0, NaN, +-inf and subnormals are exceptions (R1).
 *   R19 analytics on compressed data (Sec. 7 names it as future work and fixes nothing): an
 *       aggregate of a stream's values, count, number of NaNs, min and max of the other
 *       values in IEEE 754 totalOrder (-0 < +0; NaN when there is none) and their sum, taken
 *       from the records without writing the values out.  The oracle decompresses (Sec. 4)
 *       and aggregates by the definition; its sum is the exact sum correctly rounded to FP64
 *       (an inf of one sign gives that inf, both signs NaN).
 *   R17 the ablation variants of Sec. 5.4.2 (Fig. 12b) change one step each and keep the
 *       record layout, so the one decoder reads all of them:
 *         Fal._Sparse / Fal._Dense: every row of M^T stored sparse / dense;
 *         Fal._Elf: the decimal place of a value is the trial-and-error one of Sec. 1, the
 *         first i >= 0 with v (x) 10^i == floor(v (x) 10^i), enumerated within Alg. 2's
 *         bounds (beta <= 15, alpha <= 22; FP32 7 and 10), none found = exception; the
 *         chunk's Case decision (Eq. 4) and the R6 round-trip check are unchanged.
 *
 * Stream layout (little-endian):
 *   0  "FLCN"  4  version=1 (u8)  5  dtype (u8: 0=f64, 1=f32, 2=f16)  6  reserved u16 = 0
 *   8  block_size u32   12 reserved u32 = 0   16 n u64   24 num_chunks u64
 *   32 u32 size[num_chunks]   then the chunk records, concatenated.
 * Chunk record: [alpha_max u8][beta_hat_max u8][z_1: 8 B (f32: 4 B, f16: 2 B)][w u8]
 *               [flags: ceil(w/8) B][row 1] ... [row w]
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>
#include <math.h>

enum { OR_F64 = 0, OR_F32 = 1, OR_F16 = 2 };

static int dtype_ok(int dtype) { return dtype == OR_F64 || dtype == OR_F32 || dtype == OR_F16; }
static size_t elem_size(int dtype) { return dtype == OR_F64 ? 8 : (dtype == OR_F32 ? 4 : 2); }
/* bits per value = bit planes of M^T (64 / 32 / 16); z_1 takes width / 8 bytes (R7) */
static int width_of(int dtype) { return 8 * (int)elem_size(dtype); }
enum { OR_OK = 0, OR_ERR_INVALID = 1, OR_ERR_CAPACITY = 2, OR_ERR_CORRUPT = 3 };

#define OR_HEADER_BYTES 32u
/* Sec. 3.3 makes chunks of n = 64k + 1 values (rows of the transposed matrix byte-aligned)
   and the implementation uses n = 1025; the stream format takes n <= 1025 (k <= 16). */
#define OR_MAX_BLOCK 1025u

/* ------------------------------------------------------------------------------------ */
/* Powers of ten, correctly rounded, from the C library's decimal parser.               */
/* ------------------------------------------------------------------------------------ */
#define P10_LO (-350)
#define P10_HI 330
static double p10_64[P10_HI - P10_LO + 1];
static float p10_32[P10_HI - P10_LO + 1];
static int p10_ready = 0;

static void init_p10(void)
{
    if (p10_ready) return;
    char buf[32];
    for (int k = P10_LO; k <= P10_HI; ++k) {
        snprintf(buf, sizeof buf, "1e%d", k);
        p10_64[k - P10_LO] = strtod(buf, NULL);
        p10_32[k - P10_LO] = strtof(buf, NULL);
    }
    p10_ready = 1;
}

/* fl(10^k) in FP64 / FP32 */
double oracle_pow10_f64(int k) { init_p10(); return p10_64[k - P10_LO]; }
float oracle_pow10_f32(int k) { init_p10(); return p10_32[k - P10_LO]; }

/* ------------------------------------------------------------------------------------ */
/* Bit views                                                                            */
/* ------------------------------------------------------------------------------------ */
static uint64_t bits64(double v) { uint64_t u; memcpy(&u, &v, 8); return u; }
static double from_bits64(uint64_t u) { double v; memcpy(&v, &u, 8); return v; }
static uint32_t bits32(float v) { uint32_t u; memcpy(&u, &v, 4); return u; }
static float from_bits32(uint32_t u) { float v; memcpy(&v, &u, 4); return v; }

/* R1: special numbers (footnote of Sec. 2.1) are treated as exceptions. */
int oracle_is_special_f64(double v)
{
    uint64_t u = bits64(v);
    uint64_t e = (u >> 52) & 0x7FF;
    if (e == 0x7FF) return 1;                     /* NaN (any payload), +-inf */
    if (e == 0 && (u << 1) != 0) return 1;        /* subnormal */
    if (u == 0x8000000000000000ull) return 1;     /* -0.0 */
    return 0;
}

int oracle_is_special_f32(float v)
{
    uint32_t u = bits32(v);
    uint32_t e = (u >> 23) & 0xFF;
    if (e == 0xFF) return 1;
    if (e == 0 && (u << 1) != 0) return 1;
    if (u == 0x80000000u) return 1;
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* R3: floor(log10|v|) as the largest k with |v| >= fl(10^k). a > 0, finite, normal.    */
/* The libm estimate is only a starting point; the table decides.                      */
/* ------------------------------------------------------------------------------------ */
int oracle_floor_log10_f64(double a)
{
    init_p10();
    int k = (int)floor(log10(a));
    if (k < P10_LO + 2) k = P10_LO + 2;
    if (k > P10_HI - 2) k = P10_HI - 2;
    while (a < oracle_pow10_f64(k)) --k;
    while (a >= oracle_pow10_f64(k + 1)) ++k;
    return k;
}

int oracle_floor_log10_f32(float a)
{
    init_p10();
    int k = (int)floor(log10((double)a));
    if (k < P10_LO + 2) k = P10_LO + 2;
    if (k > P10_HI - 2) k = P10_HI - 2;
    while (a < oracle_pow10_f32(k)) --k;
    while (a >= oracle_pow10_f32(k + 1)) ++k;
    return k;
}

/* ------------------------------------------------------------------------------------ */
/* Alg. 2 DPAndDSCalculation(v) (Sec. 3.2.2): enumerate alpha from 0, stop at the first */
/* alpha with eps <= mu (Thm 4), verify the round trip (otherwise exception (23,16)).   */
/* Loop while beta <= 15 and alpha <= 22. alpha > 22 or beta > 15 means exception.      */
/* ------------------------------------------------------------------------------------ */
void oracle_dp_ds_f64(double v, int *alpha, int *beta)
{
    if (oracle_is_special_f64(v)) { *alpha = 23; *beta = 16; return; }   /* R1 */
    if (v == 0.0) { *alpha = 0; *beta = 0; return; }                     /* special case */
    int a = 0;
    int b = a + oracle_floor_log10_f64(fabs(v)) + 1;                    /* Eq. 2 */
    while (b <= 15 && a <= 22) {
        double x = v * oracle_pow10_f64(a);                             /* v (x) 10^alpha */
        double r = round(x);
        if (fabs(x - r) <= fabs(x) * 0x1p-52) {                         /* eps <= mu */
            if (r / oracle_pow10_f64(a) != v) { a = 23; b = 16; }       /* round trip */
            break;
        }
        a = a + 1;
        b = b + 1;
    }
    *alpha = a;
    *beta = b;
}

/* FP32 analogue (R14): alpha <= 10, beta <= 7, mu = |x| * 2^-23, x exact in FP64. */
void oracle_dp_ds_f32(float v, int *alpha, int *beta)
{
    if (oracle_is_special_f32(v)) { *alpha = 11; *beta = 8; return; }
    if (v == 0.0f) { *alpha = 0; *beta = 0; return; }
    int a = 0;
    int b = a + oracle_floor_log10_f32(fabsf(v)) + 1;
    while (b <= 7 && a <= 10) {
        double x = (double)v * (double)oracle_pow10_f32(a);            /* exact */
        double r = round(x);
        if (fabs(x - r) <= fabs(x) * 0x1p-23) {
            if ((float)r / oracle_pow10_f32(a) != v) { a = 11; b = 8; }
            break;
        }
        a = a + 1;
        b = b + 1;
    }
    *alpha = a;
    *beta = b;
}

/* ------------------------------------------------------------------------------------ */
/* Fal._Elf's decimal place (Sec. 1 trial-and-error, Sec. 5.4.2 ablation; R17): the first */
/* i with v (x) 10^i an integer.  1.11 gives 3 (1.11 (x) 10^2 = 111.00000000000001).     */
/* ------------------------------------------------------------------------------------ */
void oracle_dp_elf_f64(double v, int *alpha, int *beta)
{
    if (oracle_is_special_f64(v)) { *alpha = 23; *beta = 16; return; }   /* R1 */
    if (v == 0.0) { *alpha = 0; *beta = 0; return; }
    int a = 0;
    int b = a + oracle_floor_log10_f64(fabs(v)) + 1;
    while (b <= 15 && a <= 22) {
        double x = v * oracle_pow10_f64(a);                             /* v (x) 10^i */
        if (x == floor(x)) break;                                       /* integral */
        a = a + 1;
        b = b + 1;
    }
    if (a > 22 || b > 15) { a = 23; b = 16; }
    *alpha = a;
    *beta = b;
}

void oracle_dp_elf_f32(float v, int *alpha, int *beta)
{
    if (oracle_is_special_f32(v)) { *alpha = 11; *beta = 8; return; }
    if (v == 0.0f) { *alpha = 0; *beta = 0; return; }
    int a = 0;
    int b = a + oracle_floor_log10_f32(fabsf(v)) + 1;
    while (b <= 7 && a <= 10) {
        float x = v * oracle_pow10_f32(a);                              /* FP32 multiply */
        if (x == floorf(x)) break;
        a = a + 1;
        b = b + 1;
    }
    if (a > 10 || b > 7) { a = 11; b = 8; }
    *alpha = a;
    *beta = b;
}

/* ------------------------------------------------------------------------------------ */
/* FP16 (R18).  Values are binary16 bit patterns (uint16_t); arithmetic on them is done   */
/* exactly on integers and in FP64, and every binary16 result is one correctly rounded   */
/* (ties to even) conversion of an exact value.                                         */
/* ------------------------------------------------------------------------------------ */
/* exact value of a binary16 pattern */
double oracle_half_to_double(uint16_t u)
{
    const int sign = u >> 15, e = (u >> 10) & 0x1F;
    const int m = u & 0x3FF;
    double v;
    if (e == 0x1F) v = m ? NAN : INFINITY;
    else if (e == 0) v = ldexp((double)m, -24);                 /* subnormal or zero */
    else v = ldexp((double)(1024 + m), e - 25);
    return sign ? -v : v;
}

/* binary16 nearest to (-1)^neg * num / den * 2^e2 (num, den > 0; ties to even; overflow to
   infinity, gradual underflow).  The exponent is found first (2^e <= |value| < 2^(e+1)); the
   value is then divided by its quantum 2^(max(e, -14) - 10) and rounded. */
static uint16_t half_from_ratio(int neg, uint64_t num, uint64_t den, int e2)
{
    const uint16_t sbit = neg ? 0x8000u : 0u;
    if (num == 0) return sbit;
    uint64_t n = num, d = den;
    int e = e2;
    while (n < d) { n <<= 1; --e; }
    while (n >= 2 * d) { d <<= 1; ++e; }
    if (e > 15) return sbit | 0x7C00u;                          /* beyond the largest finite */
    const int qe = (e < -14 ? -14 : e) - 10;                    /* quantum 2^qe */
    uint64_t a = num, b = den;
    if (e2 - qe >= 0) a <<= (e2 - qe); else b <<= (qe - e2);
    uint64_t k = a / b;
    const uint64_t r = a % b;
    if (2 * r > b || (2 * r == b && (k & 1))) ++k;
    if (qe == -24) return sbit | (uint16_t)k;                   /* subnormal range; k = 1024 is 2^-14 */
    int ee = e;
    if (k == 2048) { k = 1024; ++ee; }
    if (ee > 15) return sbit | 0x7C00u;
    return sbit | (uint16_t)((ee + 15) << 10) | (uint16_t)(k - 1024);
}

/* fl16(10^k) */
uint16_t oracle_pow10_f16(int k)
{
    if (k > 4) return 0x7C00u;                                  /* 10^5 > 65504 */
    uint64_t p = 1;
    for (int i = 0; i < (k < 0 ? -k : k); ++i) p *= 10;
    return k >= 0 ? half_from_ratio(0, p, 1, 0) : half_from_ratio(0, 1, p, 0);
}

/* fl16(g / 10^a), g an integer, 0 <= a <= 4: Case-1 round trip and decode (R18) */
uint16_t oracle_f16_div_pow10(int32_t g, int a)
{
    uint64_t p = 1;
    for (int i = 0; i < a; ++i) p *= 10;
    const int neg = g < 0;
    const uint64_t mag = neg ? (uint64_t)(-(int64_t)g) : (uint64_t)g;
    return half_from_ratio(neg, mag, p, 0);
}

/* R1 for binary16 */
int oracle_is_special_f16(uint16_t u)
{
    const unsigned e = (u >> 10) & 0x1F;
    if (e == 0x1F) return 1;                                    /* NaN, +-inf */
    if (e == 0 && (u & 0x3FF) != 0) return 1;                   /* subnormal */
    if (u == 0x8000u) return 1;                                 /* -0 */
    return 0;
}

/* R3 for binary16: the largest k with |v| >= fl16(10^k); |v| normal, finite */
int oracle_floor_log10_f16(uint16_t u)
{
    const double a = fabs(oracle_half_to_double(u));
    int k = (int)floor(log10(a));
    while (k > -9 && a < oracle_half_to_double(oracle_pow10_f16(k))) --k;
    while (k < 4 && a >= oracle_half_to_double(oracle_pow10_f16(k + 1))) ++k;
    return k;
}

/* Alg. 2 for binary16 (R18): alpha <= 4, beta <= 3, mu = |x| * 2^-10, x exact in FP64 */
void oracle_dp_ds_f16(uint16_t v, int *alpha, int *beta)
{
    if (oracle_is_special_f16(v)) { *alpha = 5; *beta = 4; return; }
    if (v == 0) { *alpha = 0; *beta = 0; return; }
    const double vd = oracle_half_to_double(v);
    int a = 0;
    int b = a + oracle_floor_log10_f16(v) + 1;
    while (b <= 3 && a <= 4) {
        double x = vd * oracle_half_to_double(oracle_pow10_f16(a));  /* exact */
        double r = round(x);
        if (fabs(x - r) <= fabs(x) * 0x1p-10) {
            if (oracle_f16_div_pow10((int32_t)r, a) != v) { a = 5; b = 4; }
            break;
        }
        a = a + 1;
        b = b + 1;
    }
    *alpha = a;
    *beta = b;
}

/* Fal._Elf's decimal place for binary16 (R17): the first i with v (x) 10^i integral, the
   product rounded to binary16 (the IEEE multiply of the format) */
void oracle_dp_elf_f16(uint16_t v, int *alpha, int *beta)
{
    if (oracle_is_special_f16(v)) { *alpha = 5; *beta = 4; return; }
    if (v == 0) { *alpha = 0; *beta = 0; return; }
    const int e = (v >> 10) & 0x1F;
    const uint64_t sig = 1024u + (v & 0x3FFu);                  /* |v| = sig * 2^(e - 25) */
    int a = 0;
    int b = a + oracle_floor_log10_f16(v) + 1;
    while (b <= 3 && a <= 4) {
        uint64_t p = 1;
        for (int i = 0; i < a; ++i) p *= 10;
        const double x = oracle_half_to_double(half_from_ratio(0, sig * p, 1, e - 25));
        if (x == floor(x)) break;
        a = a + 1;
        b = b + 1;
    }
    if (a > 4 || b > 3) { a = 5; b = 4; }
    *alpha = a;
    *beta = b;
}

/* ------------------------------------------------------------------------------------ */
/* Zigzag (Eq. 5): Zigzag(x) = (x << 1) xor (x >> 63), arithmetic shift (R7).           */
/* ------------------------------------------------------------------------------------ */
uint64_t oracle_zigzag64(uint64_t x)
{
    return (x << 1) ^ (uint64_t)((int64_t)x >> 63);
}
uint64_t oracle_unzigzag64(uint64_t z)
{
    return (z >> 1) ^ (0 - (z & 1));
}
uint32_t oracle_zigzag32(uint32_t x)
{
    return (x << 1) ^ (uint32_t)((int32_t)x >> 31);
}
uint32_t oracle_unzigzag32(uint32_t z)
{
    return (z >> 1) ^ (0u - (z & 1u));
}
uint16_t oracle_zigzag16(uint16_t x)
{
    return (uint16_t)((uint16_t)(x << 1) ^ (uint16_t)((int16_t)x >> 15));
}
uint16_t oracle_unzigzag16(uint16_t z)
{
    return (uint16_t)((z >> 1) ^ (uint16_t)(0u - (z & 1u)));
}

/* ------------------------------------------------------------------------------------ */
/* Digit transformation of one chunk (Sec. 3.2.3, Eq. 4, Thm 5, Alg. 3 integer part).   */
/* Output: alpha_max, beta_hat_max as stored (R12 sentinels in Case 2), case flag, and  */
/* G = {g_1..g_m} as raw 64-bit words (FP32: low 32 bits).                               */
/* Returns the number of R6 firings (values that failed the Case-1 round trip).        */
/* ------------------------------------------------------------------------------------ */
static int chunk_transform_with(const void *vals, uint32_t m, int dtype, int elf,
                                int *alpha_max_out, int *beta_hat_out, int *case1_out,
                                uint64_t *g)
{
    int r6_firings = 0;
    if (dtype == OR_F64) {
        const double *v = (const double *)vals;
        /* alpha_max = max DP(v_i) via Alg. 2; v_max = max |v_i| */
        int alpha_max = 0;
        int any_exception = 0;
        double v_max = 0.0;
        for (uint32_t i = 0; i < m; ++i) {
            int a, b;
            if (elf) oracle_dp_elf_f64(v[i], &a, &b);
            else oracle_dp_ds_f64(v[i], &a, &b);
            if (a > alpha_max) alpha_max = a;
            if (a > 22 || b > 15) any_exception = 1;
        }
        /* beta_hat_max = alpha_max + floor(log10 v_max) + 1 (0 if v_max = 0); only
           meaningful when no value is special, i.e. alpha_max <= 22. */
        int beta_hat = 16;
        if (alpha_max <= 22) {
            for (uint32_t i = 0; i < m; ++i) {
                double av = fabs(v[i]);
                if (av > v_max) v_max = av;
            }
            beta_hat = (v_max == 0.0) ? 0 : alpha_max + oracle_floor_log10_f64(v_max) + 1;
        }
        int case1 = (alpha_max <= 22 && beta_hat <= 15);
        /* An exception value always forces alpha_max > 22 or beta_hat > 15 (Eq. 2). The
           oracle checks it explicitly instead of relying on that argument. */
        if (any_exception) case1 = 0;
        if (case1) {
            double p = oracle_pow10_f64(alpha_max);
            for (uint32_t i = 0; i < m; ++i) {
                double x = v[i] * p;                     /* v_i (x) 10^alpha_max */
                int64_t gi = (int64_t)llround(x);        /* g_i = round(...) */
                g[i] = (uint64_t)gi;
                double back = (double)gi / p;            /* Thm 5: g_i / 10^alpha_max */
                if (bits64(back) != bits64(v[i])) ++r6_firings;
            }
            if (r6_firings) case1 = 0;                   /* R6 */
        }
        if (!case1) {
            for (uint32_t i = 0; i < m; ++i)
                g[i] = oracle_zigzag64(bits64(v[i])); /* g_i = Zigzag(BinLong(v_i)) */
            alpha_max = 23;
            beta_hat = 16;
        }
        *alpha_max_out = alpha_max;
        *beta_hat_out = beta_hat;
        *case1_out = case1;
    } else if (dtype == OR_F16) {
        const uint16_t *v = (const uint16_t *)vals;             /* binary16 patterns (R18) */
        int alpha_max = 0;
        int any_exception = 0;
        for (uint32_t i = 0; i < m; ++i) {
            int a, b;
            if (elf) oracle_dp_elf_f16(v[i], &a, &b);
            else oracle_dp_ds_f16(v[i], &a, &b);
            if (a > alpha_max) alpha_max = a;
            if (a > 4 || b > 3) any_exception = 1;
        }
        int beta_hat = 4;
        if (alpha_max <= 4) {
            uint16_t v_max = 0;                                 /* |v| orders as its pattern */
            for (uint32_t i = 0; i < m; ++i) {
                uint16_t av = v[i] & 0x7FFFu;
                if (av > v_max) v_max = av;
            }
            beta_hat = (v_max == 0) ? 0 : alpha_max + oracle_floor_log10_f16(v_max) + 1;
        }
        int case1 = (alpha_max <= 4 && beta_hat <= 3);
        if (any_exception) case1 = 0;
        if (case1) {
            const double p = oracle_half_to_double(oracle_pow10_f16(alpha_max));
            for (uint32_t i = 0; i < m; ++i) {
                double x = oracle_half_to_double(v[i]) * p;     /* exact */
                int32_t gi = (int32_t)llround(x);
                g[i] = (uint64_t)(uint16_t)gi;
                if (oracle_f16_div_pow10(gi, alpha_max) != v[i]) ++r6_firings;
            }
            if (r6_firings) case1 = 0;
        }
        if (!case1) {
            for (uint32_t i = 0; i < m; ++i)
                g[i] = (uint64_t)oracle_zigzag16(v[i]);
            alpha_max = 5;
            beta_hat = 4;
        }
        *alpha_max_out = alpha_max;
        *beta_hat_out = beta_hat;
        *case1_out = case1;
    } else {
        const float *v = (const float *)vals;
        int alpha_max = 0;
        int any_exception = 0;
        for (uint32_t i = 0; i < m; ++i) {
            int a, b;
            if (elf) oracle_dp_elf_f32(v[i], &a, &b);
            else oracle_dp_ds_f32(v[i], &a, &b);
            if (a > alpha_max) alpha_max = a;
            if (a > 10 || b > 7) any_exception = 1;
        }
        int beta_hat = 8;
        if (alpha_max <= 10) {
            float v_max = 0.0f;
            for (uint32_t i = 0; i < m; ++i) {
                float av = fabsf(v[i]);
                if (av > v_max) v_max = av;
            }
            beta_hat = (v_max == 0.0f) ? 0 : alpha_max + oracle_floor_log10_f32(v_max) + 1;
        }
        int case1 = (alpha_max <= 10 && beta_hat <= 7);
        if (any_exception) case1 = 0;
        if (case1) {
            float p = oracle_pow10_f32(alpha_max);
            for (uint32_t i = 0; i < m; ++i) {
                double x = (double)v[i] * (double)p;     /* exact (R14) */
                int32_t gi = (int32_t)llround(x);
                g[i] = (uint64_t)(uint32_t)gi;
                float back = (float)gi / p;
                if (bits32(back) != bits32(v[i])) ++r6_firings;
            }
            if (r6_firings) case1 = 0;
        }
        if (!case1) {
            for (uint32_t i = 0; i < m; ++i)
                g[i] = (uint64_t)oracle_zigzag32(bits32(v[i]));
            alpha_max = 11;
            beta_hat = 8;
        }
        *alpha_max_out = alpha_max;
        *beta_hat_out = beta_hat;
        *case1_out = case1;
    }
    return r6_firings;
}

int oracle_chunk_transform(const void *vals, uint32_t m, int dtype,
                           int *alpha_max_out, int *beta_hat_out, int *case1_out,
                           uint64_t *g)
{
    return chunk_transform_with(vals, m, dtype, 0, alpha_max_out, beta_hat_out, case1_out, g);
}

/* The same with Fal._Elf's decimal place (R17). */
int oracle_chunk_transform_elf(const void *vals, uint32_t m, int dtype,
                               int *alpha_max_out, int *beta_hat_out, int *case1_out,
                               uint64_t *g)
{
    return chunk_transform_with(vals, m, dtype, 1, alpha_max_out, beta_hat_out, case1_out, g);
}

/* Eq. 5: z_1 = g_1, z_i = Zigzag(g_i - g_{i-1}) for i > 1 (modulo 2^64 / 2^32 / 2^16). */
void oracle_delta_zigzag(const uint64_t *g, uint32_t m, int dtype, uint64_t *z)
{
    for (uint32_t i = 0; i < m; ++i) {
        if (i == 0) {
            z[i] = g[0];
        } else if (dtype == OR_F64) {
            z[i] = oracle_zigzag64(g[i] - g[i - 1]);
        } else if (dtype == OR_F16) {
            z[i] = (uint64_t)oracle_zigzag16((uint16_t)((uint16_t)g[i] - (uint16_t)g[i - 1]));
        } else {
            z[i] = (uint64_t)oracle_zigzag32((uint32_t)g[i] - (uint32_t)g[i - 1]);
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Sec. 3.3 adaptive bit-plane encoding of Z \ {z_1} and the chunk record (Fig. 8c).    */
/* ------------------------------------------------------------------------------------ */
static int clz64(uint64_t x) { int n = 0; if (!x) return 64; while (!(x & 0x8000000000000000ull)) { x <<= 1; ++n; } return n; }

/* cols = round_up(m - 1, 64) (R11) */
static uint32_t chunk_cols(uint32_t m) { return m <= 1 ? 0 : ((m - 1 + 63) / 64) * 64; }

/* Bit of z at plane p for column c (c indexes z_{c+2}; pad columns are 0). */
static int plane_bit(const uint64_t *z, uint32_t m, uint32_t c, int p)
{
    uint32_t idx = c + 1;                 /* 0-based index of z_{c+2} */
    if (idx >= m) return 0;               /* zero pad column (R11) */
    return (int)((z[idx] >> p) & 1u);
}

/* Row storage of the record encoder: the adaptive choice of Sec. 3.3, or every row sparse
   (Fal._Sparse) or dense (Fal._Dense) as in the ablation of Sec. 5.4.2 (R17). */
enum { OR_STORE_ADAPTIVE = 0, OR_STORE_SPARSE = 1, OR_STORE_DENSE = 2 };

/* Encodes one record; returns its byte length or 0 if it does not fit in cap. */
size_t oracle_encode_z_storage(const uint64_t *z, uint32_t m, int dtype, int alpha_max, int beta_hat,
                               int storage, uint8_t *out, size_t cap)
{
    const int width = width_of(dtype);
    const int z1_bytes = width / 8;
    const uint32_t cols = chunk_cols(m);
    const uint32_t row_bytes = cols / 8;
    const uint32_t bitmap_bytes = cols / 64;

    /* w = width - min clz(z_2..z_m); clz(0) = width */
    int lead_min = width;
    for (uint32_t i = 1; i < m; ++i) {
        int lead = clz64(z[i]) - (64 - width);
        if (lead < lead_min) lead_min = lead;
    }
    const int w = width - lead_min;
    const uint32_t flag_bytes = (uint32_t)(w + 7) / 8;

    size_t pos = 0;
#define PUT(byte) do { if (pos >= cap) return 0; out[pos++] = (uint8_t)(byte); } while (0)
    PUT(alpha_max);
    PUT(beta_hat);
    for (int k = 0; k < z1_bytes; ++k) PUT((z[0] >> (8 * k)) & 0xFF);
    PUT(w);
    size_t flag_pos = pos;
    for (uint32_t k = 0; k < flag_bytes; ++k) PUT(0);

    uint8_t *row = (uint8_t *)malloc(row_bytes ? row_bytes : 1);
    for (int r = 1; r <= w; ++r) {
        int p = w - r;                            /* R8: row 1 = plane w-1 */
        /* byte j holds columns 8j..8j+7, column 8j+i at bit 7-i (R9) */
        uint32_t lambda = 0;
        for (uint32_t j = 0; j < row_bytes; ++j) {
            unsigned byte = 0;
            for (int i = 0; i < 8; ++i)
                byte |= (unsigned)plane_bit(z, m, 8 * j + i, p) << (7 - i);
            row[j] = (uint8_t)byte;
            if (byte == 0) ++lambda;              /* zero byte */
        }
        int sparse = lambda > cols / 64;          /* Sec. 3.3 criterion, tie -> dense (R10) */
        if (storage == OR_STORE_SPARSE) sparse = 1;
        if (storage == OR_STORE_DENSE) sparse = 0;
        /* flag: the last w bits of the flag bytes, row 1 first, MSB-first (R9) */
        uint32_t bitpos = flag_bytes * 8 - (uint32_t)w + (uint32_t)(r - 1);
        if (!sparse) out[flag_pos + bitpos / 8] |= (uint8_t)(0x80u >> (bitpos % 8));
        if (sparse) {
            for (uint32_t b = 0; b < bitmap_bytes; ++b) {
                unsigned bm = 0;
                for (int i = 0; i < 8; ++i)
                    if (row[8 * b + i] != 0) bm |= 0x80u >> i;
                if (pos >= cap) { free(row); return 0; }
                out[pos++] = (uint8_t)bm;
            }
            for (uint32_t j = 0; j < row_bytes; ++j)
                if (row[j] != 0) { if (pos >= cap) { free(row); return 0; } out[pos++] = row[j]; }
        } else {
            for (uint32_t j = 0; j < row_bytes; ++j) { if (pos >= cap) { free(row); return 0; } out[pos++] = row[j]; }
        }
    }
    free(row);
#undef PUT
    return pos;
}

size_t oracle_encode_z(const uint64_t *z, uint32_t m, int dtype, int alpha_max, int beta_hat,
                       uint8_t *out, size_t cap)
{
    return oracle_encode_z_storage(z, m, dtype, alpha_max, beta_hat, OR_STORE_ADAPTIVE, out, cap);
}

/* Codec variants (R17): Falcon itself and the three ablations of Sec. 5.4.2. */
enum { OR_VARIANT_FALCON = 0, OR_VARIANT_SPARSE = 1, OR_VARIANT_DENSE = 2, OR_VARIANT_ELF = 3 };

/* One chunk of a variant: Eq. 4 -> Eq. 5 -> Sec. 3.3. Returns the record length, 0 on
   overflow or an unknown variant. */
size_t oracle_encode_chunk_variant(const void *vals, uint32_t m, int dtype, int variant,
                                   uint8_t *out, size_t cap)
{
    if (variant < OR_VARIANT_FALCON || variant > OR_VARIANT_ELF) return 0;
    uint64_t *g = (uint64_t *)malloc(sizeof(uint64_t) * (m ? m : 1));
    uint64_t *z = (uint64_t *)malloc(sizeof(uint64_t) * (m ? m : 1));
    int alpha_max, beta_hat, case1;
    if (variant == OR_VARIANT_ELF) oracle_chunk_transform_elf(vals, m, dtype, &alpha_max, &beta_hat, &case1, g);
    else oracle_chunk_transform(vals, m, dtype, &alpha_max, &beta_hat, &case1, g);
    oracle_delta_zigzag(g, m, dtype, z);
    int storage = OR_STORE_ADAPTIVE;
    if (variant == OR_VARIANT_SPARSE) storage = OR_STORE_SPARSE;
    if (variant == OR_VARIANT_DENSE) storage = OR_STORE_DENSE;
    size_t len = oracle_encode_z_storage(z, m, dtype, alpha_max, beta_hat, storage, out, cap);
    free(g);
    free(z);
    return len;
}

/* One chunk: Eq. 4 -> Eq. 5 -> Sec. 3.3. Returns the record length, 0 on overflow. */
size_t oracle_encode_chunk(const void *vals, uint32_t m, int dtype, uint8_t *out, size_t cap)
{
    return oracle_encode_chunk_variant(vals, m, dtype, OR_VARIANT_FALCON, out, cap);
}

/* ------------------------------------------------------------------------------------ */
/* Stream level (Sec. 3.4, Alg. 3): header, u32 size array (R13), records.            */
/* ------------------------------------------------------------------------------------ */
static uint64_t num_chunks_of(uint64_t n, uint32_t block) { return (n + block - 1) / block; }

static size_t record_bound(uint32_t m, int dtype)
{
    const int width = width_of(dtype);
    const int z1_bytes = width / 8;
    return 2 + (size_t)z1_bytes + 1 + (size_t)(width / 8) + (size_t)width * (chunk_cols(m) / 8);
}

size_t oracle_bound(uint64_t n, int dtype, uint32_t block)
{
    if (!dtype_ok(dtype) || block < 2 || block > OR_MAX_BLOCK) return 0;
    uint64_t nc = num_chunks_of(n, block);
    size_t total = OR_HEADER_BYTES + 4 * (size_t)nc;
    if (nc == 0) return total;
    total += (size_t)(nc - 1) * record_bound(block, dtype);
    total += record_bound((uint32_t)(n - (nc - 1) * (uint64_t)block), dtype);
    return total;
}

/* Largest record of a variant: a row is at most cols/8 bytes (dense), except under
   Fal._Sparse, where a row without zero bytes takes its bitmap as well (cols/64 + cols/8). */
size_t oracle_bound_variant(uint64_t n, int dtype, uint32_t block, int variant)
{
    size_t total = oracle_bound(n, dtype, block);
    if (total == 0 || variant != 1) return total;          /* 1 = Fal._Sparse */
    const int width = width_of(dtype);
    const uint64_t nc = num_chunks_of(n, block);
    if (nc == 0) return total;
    total += (size_t)(nc - 1) * (size_t)width * (chunk_cols(block) / 64);
    total += (size_t)width * (chunk_cols((uint32_t)(n - (nc - 1) * (uint64_t)block)) / 64);
    return total;
}

static void put_u32(uint8_t *p, uint32_t x) { for (int k = 0; k < 4; ++k) p[k] = (uint8_t)(x >> (8 * k)); }
static void put_u64(uint8_t *p, uint64_t x) { for (int k = 0; k < 8; ++k) p[k] = (uint8_t)(x >> (8 * k)); }
static uint32_t get_u32(const uint8_t *p) { uint32_t x = 0; for (int k = 3; k >= 0; --k) x = (x << 8) | p[k]; return x; }
static uint64_t get_u64(const uint8_t *p) { uint64_t x = 0; for (int k = 7; k >= 0; --k) x = (x << 8) | p[k]; return x; }

static void put_header(uint8_t *out, uint64_t n, int dtype, uint32_t block, uint64_t nc)
{
    memcpy(out, "FLCN", 4);
    out[4] = 1;
    out[5] = (uint8_t)dtype;
    out[6] = 0; out[7] = 0;
    put_u32(out + 8, block);
    put_u32(out + 12, 0);
    put_u64(out + 16, n);
    put_u64(out + 24, nc);
}

int oracle_compress_variant(const void *in, uint64_t n, int dtype, uint32_t block, int variant,
                            uint8_t *out, size_t cap, size_t *out_bytes)
{
    if (!dtype_ok(dtype) || block < 2 || block > OR_MAX_BLOCK) return OR_ERR_INVALID;
    if (variant < OR_VARIANT_FALCON || variant > OR_VARIANT_ELF) return OR_ERR_INVALID;
    const size_t s = elem_size(dtype);
    const uint64_t nc = num_chunks_of(n, block);
    const size_t data_start = OR_HEADER_BYTES + 4 * (size_t)nc;
    if (cap < data_start) return OR_ERR_CAPACITY;
    put_header(out, n, dtype, block, nc);
    size_t pos = data_start;
    for (uint64_t c = 0; c < nc; ++c) {
        uint64_t first = c * block;
        uint32_t m = (uint32_t)((n - first) < block ? (n - first) : block);
        size_t len = oracle_encode_chunk_variant((const uint8_t *)in + first * s, m, dtype, variant, out + pos,
                                                 cap - pos);
        if (len == 0) return OR_ERR_CAPACITY;
        put_u32(out + OR_HEADER_BYTES + 4 * c, (uint32_t)len);
        pos += len;
    }
    *out_bytes = pos;
    return OR_OK;
}

int oracle_compress(const void *in, uint64_t n, int dtype, uint32_t block,
                    uint8_t *out, size_t cap, size_t *out_bytes)
{
    return oracle_compress_variant(in, n, dtype, block, OR_VARIANT_FALCON, out, cap, out_bytes);
}

/* Parses a stream header. */
int oracle_stream_info(const uint8_t *in, size_t in_bytes, uint64_t *n, int *dtype, uint32_t *block,
                       uint64_t *num_chunks)
{
    if (in_bytes < OR_HEADER_BYTES) return OR_ERR_CORRUPT;
    if (memcmp(in, "FLCN", 4) != 0 || in[4] != 1) return OR_ERR_CORRUPT;
    int dt = in[5];
    uint32_t b = get_u32(in + 8);
    uint64_t nn = get_u64(in + 16);
    uint64_t nc = get_u64(in + 24);
    if (!dtype_ok(dt)) return OR_ERR_CORRUPT;
    if (b < 2 || b > OR_MAX_BLOCK) return OR_ERR_CORRUPT;
    if (nc != num_chunks_of(nn, b)) return OR_ERR_CORRUPT;
    *n = nn; *dtype = dt; *block = b; *num_chunks = nc;
    return OR_OK;
}

/* Sec. 4: decode one record of m values. Returns OR_OK or OR_ERR_CORRUPT. */
int oracle_decode_chunk(const uint8_t *rec, size_t len, uint32_t m, int dtype, void *vals)
{
    const int width = width_of(dtype);
    const int z1_bytes = width / 8;
    const uint32_t cols = chunk_cols(m);
    const uint32_t row_bytes = cols / 8;
    const uint32_t bitmap_bytes = cols / 64;
    size_t pos = 0;
    if (len < (size_t)(3 + z1_bytes)) return OR_ERR_CORRUPT;
    int alpha = rec[pos++];
    int beta_hat = rec[pos++];
    uint64_t z1 = 0;
    for (int k = 0; k < z1_bytes; ++k) z1 |= (uint64_t)rec[pos++] << (8 * k);
    int w = rec[pos++];
    if (w > width) return OR_ERR_CORRUPT;
    if (m <= 1 && w != 0) return OR_ERR_CORRUPT;
    uint32_t flag_bytes = (uint32_t)(w + 7) / 8;
    if (pos + flag_bytes > len) return OR_ERR_CORRUPT;
    size_t flag_pos = pos;
    pos += flag_bytes;

    uint64_t *z = (uint64_t *)calloc(m ? m : 1, sizeof(uint64_t));
    z[0] = z1;
    for (int r = 1; r <= w; ++r) {
        int p = w - r;
        uint32_t bitpos = flag_bytes * 8 - (uint32_t)w + (uint32_t)(r - 1);
        int dense = (rec[flag_pos + bitpos / 8] >> (7 - bitpos % 8)) & 1;
        for (uint32_t j = 0; j < row_bytes; ++j) {
            unsigned byte;
            if (dense) {
                if (pos + j >= len) { free(z); return OR_ERR_CORRUPT; }
                byte = rec[pos + j];
            } else {
                /* bitmap then the non-zero bytes in row order */
                if (pos + bitmap_bytes > len) { free(z); return OR_ERR_CORRUPT; }
                int nz = (rec[pos + j / 8] >> (7 - j % 8)) & 1;
                if (!nz) {
                    byte = 0;
                } else {
                    uint32_t rank = 0;
                    for (uint32_t q = 0; q < j; ++q) rank += (rec[pos + q / 8] >> (7 - q % 8)) & 1;
                    if (pos + bitmap_bytes + rank >= len) { free(z); return OR_ERR_CORRUPT; }
                    byte = rec[pos + bitmap_bytes + rank];
                }
            }
            for (int i = 0; i < 8; ++i) {
                uint32_t c = 8 * j + (uint32_t)i;
                if (c + 1 < m && ((byte >> (7 - i)) & 1)) z[c + 1] |= (uint64_t)1 << p;
            }
        }
        if (dense) {
            pos += row_bytes;
        } else {
            uint32_t nnz = 0;
            for (uint32_t q = 0; q < row_bytes; ++q) nnz += (rec[pos + q / 8] >> (7 - q % 8)) & 1;
            pos += bitmap_bytes + nnz;
        }
        if (pos > len) { free(z); return OR_ERR_CORRUPT; }
    }
    if (pos != len) { free(z); return OR_ERR_CORRUPT; }

    /* inverse of Eq. 5: g_1 = z_1, g_i = g_{i-1} + Unzigzag(z_i) */
    if (dtype == OR_F64) {
        int case1 = (alpha <= 22 && beta_hat <= 15);                /* R12 */
        double *out = (double *)vals;
        uint64_t g = z[0];
        for (uint32_t i = 0; i < m; ++i) {
            if (i > 0) g = g + oracle_unzigzag64(z[i]);
            /* inverse of Eq. 4 */
            if (case1) out[i] = (double)(int64_t)g / oracle_pow10_f64(alpha);
            else out[i] = from_bits64(oracle_unzigzag64(g));
        }
    } else if (dtype == OR_F16) {
        int case1 = (alpha <= 4 && beta_hat <= 3);                  /* R18 */
        uint16_t *out = (uint16_t *)vals;
        uint16_t g = (uint16_t)z[0];
        for (uint32_t i = 0; i < m; ++i) {
            if (i > 0) g = (uint16_t)(g + oracle_unzigzag16((uint16_t)z[i]));
            if (case1) out[i] = oracle_f16_div_pow10((int16_t)g, alpha);
            else out[i] = oracle_unzigzag16(g);
        }
    } else {
        int case1 = (alpha <= 10 && beta_hat <= 7);
        float *out = (float *)vals;
        uint32_t g = (uint32_t)z[0];
        for (uint32_t i = 0; i < m; ++i) {
            if (i > 0) g = g + oracle_unzigzag32((uint32_t)z[i]);
            if (case1) out[i] = (float)(int32_t)g / oracle_pow10_f32(alpha);
            else out[i] = from_bits32(oracle_unzigzag32(g));
        }
    }
    free(z);
    return OR_OK;
}

int oracle_decompress(const uint8_t *in, size_t in_bytes, void *out, size_t out_cap_bytes,
                      uint64_t *n_out)
{
    uint64_t n, nc;
    int dtype;
    uint32_t block;
    int st = oracle_stream_info(in, in_bytes, &n, &dtype, &block, &nc);
    if (st != OR_OK) return st;
    const size_t s = elem_size(dtype);
    if (n > out_cap_bytes / s) return OR_ERR_CAPACITY;
    size_t data_start = OR_HEADER_BYTES + 4 * (size_t)nc;
    if (nc > (in_bytes - OR_HEADER_BYTES) / 4 || data_start > in_bytes) return OR_ERR_CORRUPT;
    size_t pos = data_start;
    for (uint64_t c = 0; c < nc; ++c) {
        uint32_t len = get_u32(in + OR_HEADER_BYTES + 4 * c);
        if (len > in_bytes - pos) return OR_ERR_CORRUPT;
        uint64_t first = c * block;
        uint32_t m = (uint32_t)((n - first) < block ? (n - first) : block);
        st = oracle_decode_chunk(in + pos, len, m, dtype, (uint8_t *)out + first * s);
        if (st != OR_OK) return st;
        pos += len;
    }
    *n_out = n;
    return OR_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Multi-threaded drivers (for timing on all host cores and for checking large inputs):  */
/* threads take contiguous chunk ranges and call the unchanged per-chunk functions above; */
/* the records are joined in chunk order, so the stream is the single-threaded one.     */
/* ------------------------------------------------------------------------------------ */
#include <pthread.h>

typedef struct {
    const uint8_t *in;
    uint64_t n, c0, c1;
    int dtype, variant;
    uint32_t block;
    uint8_t *sizes;          /* the stream's size array */
    uint8_t *buf;            /* private records of chunks c0..c1 */
    size_t cap, len;
    int status;
    uint8_t *dst;            /* phase 2: where the records go */
} mt_comp;

static void *mt_comp_encode(void *arg)
{
    mt_comp *t = (mt_comp *)arg;
    const size_t s = elem_size(t->dtype);
    size_t pos = 0;
    for (uint64_t c = t->c0; c < t->c1; ++c) {
        uint64_t first = c * t->block;
        uint32_t m = (uint32_t)((t->n - first) < t->block ? (t->n - first) : t->block);
        size_t len = oracle_encode_chunk_variant(t->in + first * s, m, t->dtype, t->variant, t->buf + pos,
                                                 t->cap - pos);
        if (len == 0) { t->status = OR_ERR_CAPACITY; return NULL; }
        put_u32(t->sizes + 4 * c, (uint32_t)len);
        pos += len;
    }
    t->len = pos;
    return NULL;
}

static void *mt_comp_place(void *arg)
{
    mt_comp *t = (mt_comp *)arg;
    memcpy(t->dst, t->buf, t->len);
    return NULL;
}

int oracle_compress_mt(const void *in, uint64_t n, int dtype, uint32_t block, int variant, int nthreads,
                       uint8_t *out, size_t cap, size_t *out_bytes)
{
    if (!dtype_ok(dtype) || block < 2 || block > OR_MAX_BLOCK) return OR_ERR_INVALID;
    if (variant < OR_VARIANT_FALCON || variant > OR_VARIANT_ELF || nthreads < 1) return OR_ERR_INVALID;
    const uint64_t nc = num_chunks_of(n, block);
    const size_t data_start = OR_HEADER_BYTES + 4 * (size_t)nc;
    if (cap < data_start) return OR_ERR_CAPACITY;
    if ((uint64_t)nthreads > nc) nthreads = nc ? (int)nc : 1;
    mt_comp *ts = (mt_comp *)calloc((size_t)nthreads, sizeof(mt_comp));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int st = OR_OK;
    for (int i = 0; i < nthreads; ++i) {
        mt_comp *t = &ts[i];
        t->in = (const uint8_t *)in; t->n = n; t->dtype = dtype; t->variant = variant; t->block = block;
        t->c0 = nc * (uint64_t)i / (uint64_t)nthreads;
        t->c1 = nc * (uint64_t)(i + 1) / (uint64_t)nthreads;
        t->sizes = out + OR_HEADER_BYTES;
        t->cap = 0;
        for (uint64_t c = t->c0; c < t->c1; ++c) {
            uint64_t first = c * block;
            t->cap += record_bound((uint32_t)((n - first) < block ? (n - first) : block), dtype);
        }
        t->buf = (uint8_t *)malloc(t->cap ? t->cap : 1);
        if (!t->buf) st = OR_ERR_CAPACITY;
    }
    if (st == OR_OK) {
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, mt_comp_encode, &ts[i]);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        size_t pos = data_start;
        for (int i = 0; i < nthreads; ++i) {
            if (ts[i].status) st = ts[i].status;
            ts[i].dst = out + pos;
            pos += ts[i].len;
        }
        if (st == OR_OK && pos > cap) st = OR_ERR_CAPACITY;
        if (st == OR_OK) {
            for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, mt_comp_place, &ts[i]);
            for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
            put_header(out, n, dtype, block, nc);
            *out_bytes = pos;
        }
    }
    for (int i = 0; i < nthreads; ++i) free(ts[i].buf);
    free(ts);
    free(th);
    return st;
}

typedef struct {
    const uint8_t *in;
    const size_t *offs;      /* record offset of every chunk */
    uint64_t n, c0, c1;
    uint32_t block;
    int dtype, status;
    uint8_t *out;
} mt_dec;

static void *mt_dec_run(void *arg)
{
    mt_dec *t = (mt_dec *)arg;
    const size_t s = elem_size(t->dtype);
    for (uint64_t c = t->c0; c < t->c1; ++c) {
        uint64_t first = c * t->block;
        uint32_t m = (uint32_t)((t->n - first) < t->block ? (t->n - first) : t->block);
        int st = oracle_decode_chunk(t->in + t->offs[c], t->offs[c + 1] - t->offs[c], m, t->dtype, t->out + first * s);
        if (st != OR_OK) { t->status = st; return NULL; }
    }
    return NULL;
}

int oracle_decompress_mt(const uint8_t *in, size_t in_bytes, void *out, size_t out_cap_bytes, uint64_t *n_out,
                         int nthreads)
{
    uint64_t n, nc;
    int dtype;
    uint32_t block;
    if (nthreads < 1) return OR_ERR_INVALID;
    int st = oracle_stream_info(in, in_bytes, &n, &dtype, &block, &nc);
    if (st != OR_OK) return st;
    const size_t s = elem_size(dtype);
    if (n > out_cap_bytes / s) return OR_ERR_CAPACITY;
    if (nc > (in_bytes - OR_HEADER_BYTES) / 4) return OR_ERR_CORRUPT;
    size_t *offs = (size_t *)malloc(sizeof(size_t) * (size_t)(nc + 1));
    if (!offs) return OR_ERR_CAPACITY;
    offs[0] = OR_HEADER_BYTES + 4 * (size_t)nc;
    for (uint64_t c = 0; c < nc; ++c) {
        uint32_t len = get_u32(in + OR_HEADER_BYTES + 4 * c);
        if (len > in_bytes - offs[c]) { free(offs); return OR_ERR_CORRUPT; }
        offs[c + 1] = offs[c] + len;
    }
    if ((uint64_t)nthreads > nc) nthreads = nc ? (int)nc : 1;
    mt_dec *ts = (mt_dec *)calloc((size_t)nthreads, sizeof(mt_dec));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int i = 0; i < nthreads; ++i) {
        mt_dec *t = &ts[i];
        t->in = in; t->offs = offs; t->n = n; t->block = block; t->dtype = dtype; t->out = (uint8_t *)out;
        t->c0 = nc * (uint64_t)i / (uint64_t)nthreads;
        t->c1 = nc * (uint64_t)(i + 1) / (uint64_t)nthreads;
        pthread_create(&th[i], NULL, mt_dec_run, t);
    }
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    st = OR_OK;
    for (int i = 0; i < nthreads; ++i) if (ts[i].status) { st = ts[i].status; break; }
    free(ts);
    free(th);
    free(offs);
    if (st == OR_OK) *n_out = n;
    return st;
}

/* ------------------------------------------------------------------------------------ */
/* R19: aggregate of a stream's values, by decompressing it (Sec. 4) and applying the     */
/* definition.  The sum of the non-NaN values is exact, then rounded once: the values are */
/* kept as a list of non-overlapping FP64 partials whose exact sum is the running total  */
/* (each addition split into its rounded sum and its error by the two-sum of Knuth, TAOCP */
/* Vol. 2, 4.2.2; the partial list as in Shewchuk, "Adaptive Precision Floating-Point    */
/* Arithmetic", 1997), and the partials are added once at the end with the rounding      */
/* corrected (half-way cases resolved by the next partial).                              */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double *p;
    size_t n, cap;
} exact_sum;

static void exact_add(exact_sum *s, double x)
{
    size_t k = 0;
    for (size_t i = 0; i < s->n; ++i) {
        double y = s->p[i];
        if (fabs(x) < fabs(y)) { double t = x; x = y; y = t; }
        const double hi = x + y;
        const double lo = y - (hi - x);                /* exact, |x| >= |y| */
        if (lo != 0.0) s->p[k++] = lo;
        x = hi;
    }
    if (k >= s->cap) {
        s->cap = 2 * s->cap + 8;
        s->p = (double *)realloc(s->p, sizeof(double) * s->cap);
    }
    s->p[k++] = x;
    s->n = k;
}

static double exact_result(const exact_sum *s)
{
    if (s->n == 0) return 0.0;
    size_t i = s->n - 1;
    double hi = s->p[i], lo = 0.0;
    while (i > 0) {
        const double x = hi, y = s->p[--i];
        hi = x + y;
        const double yr = hi - x;
        lo = y - yr;
        if (lo != 0.0) break;
    }
    /* the rounding of hi is exact to half an ulp; a half-way case with more partials below
       of the same sign as lo rounds away from hi */
    if (i > 0 && ((lo < 0.0 && s->p[i - 1] < 0.0) || (lo > 0.0 && s->p[i - 1] > 0.0))) {
        const double y = lo * 2.0, x = hi + y, yr = x - hi;
        if (y == yr) hi = x;
    }
    return hi;
}

static uint64_t total_order_key(double v)
{
    const uint64_t b = bits64(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

int oracle_aggregate(const uint8_t *in, size_t in_bytes, uint64_t *count, uint64_t *nan_count, double *vmin,
                     double *vmax, double *sum)
{
    uint64_t n, nc;
    int dtype;
    uint32_t block;
    int st = oracle_stream_info(in, in_bytes, &n, &dtype, &block, &nc);
    if (st != OR_OK) return st;
    const size_t s = elem_size(dtype);
    uint8_t *vals = (uint8_t *)malloc(n ? n * s : 1);
    if (!vals) return OR_ERR_CAPACITY;
    uint64_t got = 0;
    st = oracle_decompress(in, in_bytes, vals, n * s, &got);
    if (st != OR_OK) { free(vals); return st; }
    exact_sum es = {NULL, 0, 0};
    uint64_t nans = 0, kmin = 0, kmax = 0;
    int any = 0, pinf = 0, ninf = 0;
    double lo = NAN, hi = NAN;
    for (uint64_t i = 0; i < n; ++i) {
        double v;
        if (dtype == OR_F64) { memcpy(&v, vals + 8 * i, 8); }
        else if (dtype == OR_F32) { float f; memcpy(&f, vals + 4 * i, 4); v = (double)f; }
        else { uint16_t h; memcpy(&h, vals + 2 * i, 2); v = oracle_half_to_double(h); }
        if (isnan(v)) { ++nans; continue; }
        const uint64_t k = total_order_key(v);
        if (!any || k < kmin) { kmin = k; lo = v; }
        if (!any || k > kmax) { kmax = k; hi = v; }
        any = 1;
        if (isinf(v)) { if (v > 0) pinf = 1; else ninf = 1; }
        else exact_add(&es, v);
    }
    double total = exact_result(&es);
    if (pinf && ninf) total = NAN;
    else if (pinf) total = INFINITY;
    else if (ninf) total = -INFINITY;
    free(es.p);
    free(vals);
    *count = n;
    *nan_count = nans;
    *vmin = lo;
    *vmax = hi;
    *sum = total;
    return OR_OK;
}

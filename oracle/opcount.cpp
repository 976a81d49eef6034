/*
 * Op-counting build of the FP64 oracle -- TEST AND MEASUREMENT INFRASTRUCTURE ONLY (used by the
 * benchmark's roofline figures; the CUDA library never calls it and shares no code with it).
 *
 * The oracle's own source (helios_ref.c) is compiled here as C++ with its floating-point type
 * replaced by `cnum`, a double that counts every arithmetic operation performed on it and
 * carries one flag: whether the value depends on the radiation field.  The flag is set on the
 * two inputs the fluxes come from (T_irr, the incident flux of eq. 20, and T_int, the internal
 * flux of eq. 22) and on the warm-start fluxes, and it propagates through every operation.
 * Operations on unflagged values (opacities, optical depths, transmissions, two-stream
 * coefficients, Planck values) are the layer coefficients of the method; operations on flagged
 * values are the flux recurrences and sums.  The counts are those of the formulas as the oracle
 * writes them, so they do not depend on how the CUDA path is organised.
 *
 * A quotient of a field-dependent value by a field-independent one counts as a multiplication on
 * the field and a division (the reciprocal) among the coefficients.
 *
 * Categories: additions/subtractions, multiplications, divisions, exponentials (exp, expm1),
 * square roots, logarithms (log, log10, log1p) and powers (pow).  Negation, absolute value,
 * comparisons, floor and conversions are not counted.  Counting is single-threaded (the
 * oracle's OpenMP pragmas are ignored in this build).
 */
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>

enum { OPC_ADD, OPC_MUL, OPC_DIV, OPC_EXP, OPC_SQRT, OPC_LOG, OPC_POW, OPC_NCAT };

static long long g_ops[2][OPC_NCAT];   // [depends on the radiation field][category]

struct cnum {
    double v;
    unsigned char f;                 // 1: depends on the radiation field
    unsigned char pad[7];
    cnum() : v(0.0), f(0) {}
    cnum(double x) : v(x), f(0) {}
    cnum(float x) : v(x), f(0) {}
    cnum(int x) : v(x), f(0) {}
    cnum(long x) : v((double)x), f(0) {}
    cnum(long long x) : v((double)x), f(0) {}
    cnum(unsigned x) : v(x), f(0) {}
    cnum(unsigned long x) : v((double)x), f(0) {}
    explicit operator int() const { return (int)v; }
    explicit operator long() const { return (long)v; }
    explicit operator long long() const { return (long long)v; }
    explicit operator double() const { return v; }
};
static_assert(sizeof(cnum) == 16, "cnum layout: double value, flag byte, padding");

static inline cnum mk(double v, unsigned char f) { cnum r; r.v = v; r.f = f; return r; }
static inline cnum op2(int cat, const cnum& a, const cnum& b, double v)
{
    const unsigned char f = a.f | b.f;
    ++g_ops[f][cat];
    return mk(v, f);
}
static inline cnum op1(int cat, const cnum& a, double v)
{
    ++g_ops[a.f][cat];
    return mk(v, a.f);
}

static inline cnum operator+(const cnum& a, const cnum& b) { return op2(OPC_ADD, a, b, a.v + b.v); }
static inline cnum operator-(const cnum& a, const cnum& b) { return op2(OPC_ADD, a, b, a.v - b.v); }
static inline cnum operator*(const cnum& a, const cnum& b) { return op2(OPC_MUL, a, b, a.v * b.v); }
// a quotient of a field-dependent value by a field-independent one is, algorithmically, a
// multiplication by a coefficient's reciprocal: a multiply on the field and a reciprocal among the
// coefficients (formed once per evaluation like every other coefficient)
static inline cnum operator/(const cnum& a, const cnum& b)
{
    if (a.f && !b.f) {
        ++g_ops[0][OPC_DIV];
        ++g_ops[1][OPC_MUL];
        return mk(a.v / b.v, 1);
    }
    return op2(OPC_DIV, a, b, a.v / b.v);
}
static inline cnum operator-(const cnum& a) { return mk(-a.v, a.f); }
static inline cnum operator+(const cnum& a) { return a; }
static inline cnum& operator+=(cnum& a, const cnum& b) { a = a + b; return a; }
static inline cnum& operator-=(cnum& a, const cnum& b) { a = a - b; return a; }
static inline cnum& operator*=(cnum& a, const cnum& b) { a = a * b; return a; }
static inline cnum& operator/=(cnum& a, const cnum& b) { a = a / b; return a; }
static inline bool operator<(const cnum& a, const cnum& b) { return a.v < b.v; }
static inline bool operator>(const cnum& a, const cnum& b) { return a.v > b.v; }
static inline bool operator<=(const cnum& a, const cnum& b) { return a.v <= b.v; }
static inline bool operator>=(const cnum& a, const cnum& b) { return a.v >= b.v; }
static inline bool operator==(const cnum& a, const cnum& b) { return a.v == b.v; }
static inline bool operator!=(const cnum& a, const cnum& b) { return a.v != b.v; }

static inline cnum exp(const cnum& a) { return op1(OPC_EXP, a, std::exp(a.v)); }
static inline cnum expm1(const cnum& a) { return op1(OPC_EXP, a, std::expm1(a.v)); }
static inline cnum sqrt(const cnum& a) { return op1(OPC_SQRT, a, std::sqrt(a.v)); }
static inline cnum log(const cnum& a) { return op1(OPC_LOG, a, std::log(a.v)); }
static inline cnum log10(const cnum& a) { return op1(OPC_LOG, a, std::log10(a.v)); }
static inline cnum log1p(const cnum& a) { return op1(OPC_LOG, a, std::log1p(a.v)); }
static inline cnum pow(const cnum& a, const cnum& b) { return op2(OPC_POW, a, b, std::pow(a.v, b.v)); }
static inline cnum cos(const cnum& a) { return mk(std::cos(a.v), a.f); }
static inline cnum fabs(const cnum& a) { return mk(std::fabs(a.v), a.f); }
static inline cnum floor(const cnum& a) { return mk(std::floor(a.v), a.f); }
static inline cnum fmin(const cnum& a, const cnum& b) { return mk(std::fmin(a.v, b.v), a.f | b.f); }
static inline cnum fmax(const cnum& a, const cnum& b) { return mk(std::fmax(a.v, b.v), a.f | b.f); }
static inline bool isfinite(const cnum& a) { return std::isfinite(a.v); }
static inline bool isnan(const cnum& a) { return std::isnan(a.v); }

#define double cnum
#include "helios_ref.c"
#undef double

extern "C" {

/* Counts since the last reset: out[flag * OPC_NCAT + category]. */
void ref_opcount_get(long long* out)
{
    for (int f = 0; f < 2; ++f)
        for (int c = 0; c < OPC_NCAT; ++c) out[f * OPC_NCAT + c] = g_ops[f][c];
}

void ref_opcount_reset(void) { std::memset(g_ops, 0, sizeof g_ops); }

int ref_opcount_categories(void) { return OPC_NCAT; }

}

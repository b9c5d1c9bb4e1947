// Operation-counting build of the FP64 oracle (TEST INFRASTRUCTURE ONLY, like oracle.c):
// oracle.c compiled as C++ with its scalar `real` a double-sized type that performs each
// operation in double and counts it, by the phase of the algorithm (ORC_PHASE markers in
// oracle.c) and kind: additions and subtractions, multiplications, divisions, square
// roots, elementary functions (sin, cos, atan2, exp, log), and comparisons / abs / min /
// max (not floating-point work). An operation whose result is fixed by a structural
// operand (an added or subtracted 0, a factor 0 or +-1, a divisor +-1, a dividend 0) is
// also counted as trivial. The result is the work of the algorithm as the oracle
// specifies it: dense 6x6 spatial algebra, model constants (body inertias) recomputed each
// step. Only the tests load it.
#include <math.h>
#include <string.h>

#define ORC_COUNTING 1

enum { OP_ADD, OP_MUL, OP_DIV, OP_SQRT, OP_FUNC, OP_CMP, OP_TADD, OP_TMUL, OP_TDIV, OP_NKINDS };

static int orc_count_phase = 0;
static double orc_counts[16][OP_NKINDS];

static inline void tally(int kind, bool trivial) {
    orc_counts[orc_count_phase][kind] += 1.0;
    if (trivial) orc_counts[orc_count_phase][kind == OP_ADD ? OP_TADD : (kind == OP_MUL ? OP_TMUL : OP_TDIV)] += 1.0;
}

struct creal {
    double v;
    creal() = default;
    creal(double x) : v(x) {}
    explicit operator double() const { return v; }
    explicit operator int() const { return (int)v; }
    creal& operator+=(creal b);
    creal& operator-=(creal b);
    creal& operator*=(creal b);
    creal& operator/=(creal b);
};
static_assert(sizeof(creal) == sizeof(double) && alignof(creal) == alignof(double), "layout of double");

static inline bool unit(double x) { return x == 1.0 || x == -1.0; }
static inline creal operator+(creal a, creal b) { tally(OP_ADD, a.v == 0.0 || b.v == 0.0); return creal(a.v + b.v); }
static inline creal operator-(creal a, creal b) { tally(OP_ADD, a.v == 0.0 || b.v == 0.0); return creal(a.v - b.v); }
static inline creal operator*(creal a, creal b) {
    tally(OP_MUL, a.v == 0.0 || b.v == 0.0 || unit(a.v) || unit(b.v));
    return creal(a.v * b.v);
}
static inline creal operator/(creal a, creal b) { tally(OP_DIV, a.v == 0.0 || unit(b.v)); return creal(a.v / b.v); }
static inline creal operator-(creal a) { return creal(-a.v); }   // a sign flip, not counted
static inline creal operator+(creal a) { return a; }
inline creal& creal::operator+=(creal b) { *this = *this + b; return *this; }
inline creal& creal::operator-=(creal b) { *this = *this - b; return *this; }
inline creal& creal::operator*=(creal b) { *this = *this * b; return *this; }
inline creal& creal::operator/=(creal b) { *this = *this / b; return *this; }
#define ORC_CMP(op)                                                                     \
    static inline bool operator op(creal a, creal b) { tally(OP_CMP, false); return a.v op b.v; }
ORC_CMP(<)
ORC_CMP(>)
ORC_CMP(<=)
ORC_CMP(>=)
ORC_CMP(==)
ORC_CMP(!=)
#undef ORC_CMP
static inline creal sqrt(creal a) { tally(OP_SQRT, false); return creal(::sqrt(a.v)); }
static inline creal sin(creal a) { tally(OP_FUNC, false); return creal(::sin(a.v)); }
static inline creal cos(creal a) { tally(OP_FUNC, false); return creal(::cos(a.v)); }
static inline creal exp(creal a) { tally(OP_FUNC, false); return creal(::exp(a.v)); }
static inline creal log(creal a) { tally(OP_FUNC, false); return creal(::log(a.v)); }
static inline creal atan2(creal a, creal b) { tally(OP_FUNC, false); return creal(::atan2(a.v, b.v)); }
static inline creal fabs(creal a) { tally(OP_CMP, false); return creal(::fabs(a.v)); }
static inline creal fmin(creal a, creal b) { tally(OP_CMP, false); return creal(::fmin(a.v, b.v)); }
static inline creal fmax(creal a, creal b) { tally(OP_CMP, false); return creal(::fmax(a.v, b.v)); }
static inline bool isfinite(creal a) { return ::isfinite(a.v); }

typedef creal real;
#define ORC_PHASE(p) (orc_count_phase = (p))

#include "oracle.c"

extern "C" {
// Counts of one rollout of one sample (H steps, knots [nk][2][nu], orc_rollout_ex): out
// [PH_COUNT][OP_NKINDS] (phase-major). Returns the rollout's cost.
double orc_count_rollout(const orc_model* m, const double* x0, const double* knots, int nk, int H, double dt,
                         int spline, double* out) {
    memset(orc_counts, 0, sizeof orc_counts);
    orc_count_phase = PH_OTHER;
    const creal S = orc_rollout_ex(m, reinterpret_cast<const creal*>(x0), reinterpret_cast<const creal*>(knots), nk, H,
                                   creal(dt), spline, nullptr, nullptr);
    for (int p = 0; p < PH_COUNT; ++p)
        for (int k = 0; k < OP_NKINDS; ++k) out[p * OP_NKINDS + k] = orc_counts[p][k];
    return S.v;
}
int orc_count_dims(int* out) {
    out[0] = PH_COUNT;
    out[1] = OP_NKINDS;
    return 0;
}
}

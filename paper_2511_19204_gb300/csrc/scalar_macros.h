// Scalar type of the chain rollout bodies (rollout_lanes.cuh, rollout_split.cuh): R_T and
// its literals and elementary functions. The FP32 product (R_DOUBLE undefined) spells
// them exactly as the bodies were written for float: the same tokens after preprocessing,
// so the same machine code; the FP64 check build (R_DOUBLE defined) maps them to double
// and to the library's correctly rounded functions. Included once per instantiation,
// right before the bodies; it redefines everything it defines.
#undef R_T
#undef R_C
#undef R_FMA
#undef R_SQRT
#undef R_RSQRT
#undef R_MAX
#undef R_ABS
#undef R_FDIV
#undef R_SINCOS
#undef R_ATAN2P
#undef R_PIN
#undef R_NS_BEGIN
#undef R_NS_END
#ifndef R_DOUBLE
#define R_T float
#define R_C(x) x##f
#define R_FMA fmaf
#define R_SQRT sqrtf
#define R_RSQRT rsqrtf
#define R_MAX fmaxf
#define R_ABS fabsf
#define R_FDIV __fdividef
#define R_SINCOS fast_sincos
#define R_ATAN2P fast_atan2_pos
#define R_PIN "+f"
#define R_NS_BEGIN namespace mppi {
#define R_NS_END }
#else
#define R_T double
#define R_C(x) x
#define R_FMA fma
#define R_SQRT sqrt
#define R_RSQRT(x) (1.0 / sqrt(x))
#define R_MAX fmax
#define R_ABS fabs
#define R_FDIV(a, b) ((a) / (b))
#define R_SINCOS sincos
#define R_ATAN2P atan2
#define R_PIN "+d"
#define R_NS_BEGIN namespace mppi { namespace f64 {
#define R_NS_END } }
#endif

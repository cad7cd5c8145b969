/*
 * repro_oracle.c -- CPU oracle for the reproducible grouped SUM repro<T,L>
 * of Mueller, Arteaga, Hoefler, Alonso, "Reproducible Floating-Point
 * Aggregation in RDBMSs" (arXiv 1802.09883).
 *
 * TEST INFRASTRUCTURE ONLY: built and called by tests/, by
 * __graft_entry__.smoke() and by the CPU-baseline leg of bench.py.  The
 * library's CUDA path neither links nor calls it, and shares no code with it.
 *
 * It follows the paper's algorithm in the paper's own representation: the
 * state of a group is repro<T,L> = <S[L], C[L]> (Sec. IV), each value is
 * added by one iteration of Algorithm 2 (RSum Scalar: check extractor
 * validity and raise levels, transform level by level, carry-bit
 * propagation), states merge with operator+=(repro) (Sec. V-B, eq. (2)/(3))
 * and the result is eq. (1).  Arithmetic is IEEE double / float in round to
 * nearest even; build with -ffp-contract=off so no multiply-add is fused.
 *
 * Readings of the paper (the exact model in exact.py lists them as R1..R7):
 * raise threshold 2^(W-1) ulp(S^(1)) as listed (R1); extraction against the
 * constant extractor 1.5 ufp(S^(l)) (R2); levels on the global grid
 * u(k) = 2^(g_min + k W), g_min = -1074 (double) / -149 (float) (R3), so the
 * initial state is the window at grid index 0 and levels below grid index 0
 * are absent; exact integer carry counts (R4); NaN / Inf / out-of-range
 * values flagged (R5); eq. (1) folded from the last level (R6); merges align
 * to the larger window (R7).
 *
 * Limits: eq. (1) is evaluated exactly while every level's exact integer
 * stays below 2^53 in magnitude (n < 2^13 values at full digit size, far
 * more in practice); the tests stay inside that range.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LMAX 4
#define ORC_FLAG_NAN 1u
#define ORC_FLAG_POS_INF 2u
#define ORC_FLAG_NEG_INF 4u
#define ORC_FLAG_RANGE 8u

#define OT_MAX_f64 DBL_MAX
#define OT_MAX_f32 FLT_MAX

/* double: m = 52, W = 40, g_min = -1074, top grid index 51 */
#define OT double
#define OSUF f64
#define OM 52
#define OW 40
#define OGMIN (-1074)
#define OKMAX 51
#define OFREXP frexp
#define OLDEXP ldexp
#define OFABS fabs
#define OFLOOR floor
#include "repro_oracle_body.h"
#undef OT
#undef OSUF
#undef OM
#undef OW
#undef OGMIN
#undef OKMAX
#undef OFREXP
#undef OLDEXP
#undef OFABS
#undef OFLOOR

/* float: m = 23, W = 18, g_min = -149, top grid index 14 */
#define OT float
#define OSUF f32
#define OM 23
#define OW 18
#define OGMIN (-149)
#define OKMAX 14
#define OFREXP frexpf
#define OLDEXP ldexpf
#define OFABS fabsf
#define OFLOOR floorf
#include "repro_oracle_body.h"

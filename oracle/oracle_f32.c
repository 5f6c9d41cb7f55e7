/*
 * The oracle's path tracer evaluated in single precision (test infrastructure only): the same
 * source as oracle.c with its floating-point type narrowed to float, so that the tests can tell a
 * path whose radiance FP32 arithmetic cannot resolve to the parity tolerance (its FP32 evaluation
 * already differs from the FP64 one) from a path where the CUDA path differs for another reason.
 * Literal constants stay double, so some intermediate products are wider than float; the
 * classification needs only that the evaluation carries FP32 rounding of every stored value.
 * It is never a reference value: every expected value comes from the FP64 build.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define double float
#include "oracle.c"

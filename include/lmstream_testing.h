/*
 * lmstream_testing.h - exports of liblmstream that exist for tests only.
 * They are not part of the stream API (include/lmstream.h); applications
 * should not call them.
 */
#ifndef LMSTREAM_TESTING_H
#define LMSTREAM_TESTING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The floor division the kernels use for pane ids, exposed so that host tests
 * can check it: returns n / d for d >= 1 computed by the invariant
 * multiply-and-shift method of Granlund & Montgomery (1994); 0 for d == 0. */
uint64_t lms_udiv_invariant(uint64_t n, uint64_t d);

#ifdef __cplusplus
}
#endif

#endif /* LMSTREAM_TESTING_H */

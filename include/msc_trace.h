/*
 * msc_trace.h -- launch counting and per-kernel device timing for libmsc.
 *
 * The paper has no counterpart (it reports wall-clock tables only); these
 * calls exist so that a caller can see which kernels a call launched and
 * how long each took on the device.
 *
 *  - msc_launch_count: total number of kernels libmsc has launched in this
 *    process (monotonic; host-side counter, no GPU work).
 *  - msc_trace_enable(on): while on, every libmsc kernel launch is
 *    bracketed by two CUDA events on its stream (events come from a pool
 *    the library owns; recording them adds a few microseconds of host time
 *    per launch).
 *  - msc_trace_reset: forget recorded launches and recycle the events.
 *  - msc_trace_collect(buf, cap): wait for the recorded events and write a
 *    JSON object {"label": [launches, total_ms], ...} (NUL-terminated) into
 *    the host buffer `buf` of `cap` bytes.  Returns MSC_OK, MSC_ERR_ARG when
 *    `cap` is too small, MSC_ERR_CUDA when an event query fails.
 * Not thread-safe with respect to concurrent collect/reset; recording from
 * several host threads is serialised internally.
 */
#ifndef MSC_TRACE_H
#define MSC_TRACE_H

#include <stddef.h>

#include "msc.h"

#ifdef __cplusplus
extern "C" {
#endif

MSC_API unsigned long long msc_launch_count(void);
MSC_API void msc_trace_enable(int on);
MSC_API void msc_trace_reset(void);
MSC_API int msc_trace_collect(char* buf, size_t cap);

#ifdef __cplusplus
}
#endif

#endif /* MSC_TRACE_H */

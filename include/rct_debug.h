/*
 * rct_debug.h -- debugging hooks of librct.so (not needed to use the library).
 *
 * Bounds-checking build: the library compiled with -DRCT_CHECK_BOUNDS (the
 * Python binding builds and loads it when RCT_BUILD_VARIANT=check).  Before
 * every access, each computed index of a staged image, of a plain-load tap
 * and of the volume is checked against its buffer; a violation is counted on
 * the device and the access skipped (no trap).  This stands in for a memory
 * checker: a run that reports zero violations made no out-of-bounds access.
 * The paper has no counterpart.
 */
#ifndef RCT_DEBUG_H
#define RCT_DEBUG_H

#include "rct.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * The context's violation count.  Waits for the context's queued work first
 * (not for other contexts').  RCT_ENOTSUP from the normal build; RCT_EINVAL
 * for a null pointer.
 */
RCT_API rct_status rct_debug_bound_violations(rct_ctx *ctx, unsigned long long *count);

/*
 * Checking build only: compare staged-image indices against at most
 * staged_elems elements (0 restores the real size), so that in-bounds
 * accesses past that limit are counted and skipped -- a control that the
 * checks are live.  No access leaves its buffer.  RCT_ENOTSUP from the normal
 * build; RCT_EINVAL for a negative limit.
 */
RCT_API rct_status rct_debug_lower_bound_limit(rct_ctx *ctx, long long staged_elems);

#ifdef __cplusplus
}
#endif

#endif /* RCT_DEBUG_H */

// Library-internal entry points of librve (not part of the public C ABI in include/rve.h;
// hidden from the shared library's exported symbols), used by the serving layer.
#pragma once
#include "../../include/rve.h"

#define RVE_INTERNAL __attribute__((visibility("hidden")))

#ifdef __cplusplus
extern "C" {
#endif

// Launch groups for handles advanced concurrently by different host threads: a handle joins a
// group of handles of its shape, precision and tiles after creation (tuning its tiles first if
// needed) and leaves it before it is destroyed; while it is a member, its BiCGStab chunks run
// as grouped launches with the other members' (results identical to running alone).
RVE_INTERNAL void *rve_group_pool_create(void);
RVE_INTERNAL void rve_group_pool_destroy(void *pool);
RVE_INTERNAL int rve_group_pool_join(void *pool, rve_t *h);
RVE_INTERNAL void rve_group_pool_leave(void *pool, rve_t *h);

#ifdef __cplusplus
}
#endif

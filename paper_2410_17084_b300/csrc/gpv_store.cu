// gpv_store.cu -- device voxel store (supplementary Alg. 2).  Placeholder sizes until
// the serving path is built; a handle without a store (hash_capacity = 0) needs none.
#include "gpv_store.h"

struct gpv_store {
    int unused;
};

size_t store_bytes(const gp_voxels_config* c) { return c->hash_capacity ? 0 : 0; }

int store_create(const gp_voxels_config*, gpv_store** out, size_t*)
{
    *out = nullptr;
    return GPV_EINVAL;
}

void store_destroy(gpv_store* s) { delete s; }

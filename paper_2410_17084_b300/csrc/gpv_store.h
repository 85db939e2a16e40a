// gpv_store.h -- device voxel store of ALG.STORE / ALG.HASH (supplementary Alg. 2):
// an open-addressing hash from voxel key to slot, a capped point bucket per slot and
// the per-scan list of visited voxels (S_updated).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/gp_voxels.h"

struct gpv_store;

size_t store_bytes(const gp_voxels_config* c);
int store_create(const gp_voxels_config* c, gpv_store** out, size_t* bytes_acc);
void store_destroy(gpv_store* s);

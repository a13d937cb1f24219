// tcgen05 tensor-core Schur update on exact 8-bit limbs (placeholder unit).
#include "cup_internal.cuh"

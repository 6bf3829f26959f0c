// muca_full_48.cu - whole-sweep kernels for L = 48.
#define MUCA_L 48
#include "muca_full.cuh"

// Device-side includes of the precompiled kernels.
#pragma once

#include <cstdint>
#include <cuda.h>

#include "kernels.h"
#include "ptx_common.cuh"

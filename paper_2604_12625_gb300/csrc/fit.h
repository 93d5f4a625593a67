// Differentiable fit: declarations used by the C ABI layer.
#pragma once
#include "ndgi_internal.h"

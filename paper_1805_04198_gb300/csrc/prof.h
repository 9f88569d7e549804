// prof.h -- optional event bracketing of kernel launches (eik_profile_*).
#pragma once

#include <cuda_runtime.h>

namespace eik {

// Returns a token to pass to prof_end, or -1 when profiling is off.
int prof_begin(const char *name, cudaStream_t s);
void prof_end(int token, cudaStream_t s);

// Brackets one launch expression.
#define EIK_LAUNCH(name, stream, ...)                 \
    do {                                              \
        int eik_tok_ = ::eik::prof_begin(name, stream); \
        __VA_ARGS__;                                  \
        ::eik::prof_end(eik_tok_, stream);            \
    } while (0)

}  // namespace eik

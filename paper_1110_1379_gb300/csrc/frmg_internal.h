// frmg_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>

struct frmg_ctx;

// cached device allocation; throws (the solver's error type) when the device
// is out of memory, so callers in other translation units catch (...)
void *frmg_alloc(frmg_ctx *c, size_t bytes);
// the context's pinned host buffer of at least n doubles (null on failure)
double *frmg_pinned(frmg_ctx *c, size_t n);
void frmg_release(frmg_ctx *c, void *p);
void frmg_set_error(const std::string &s);
long long &frmg_launch_counter(frmg_ctx *c);
// the device a context was created on
int frmg_device(frmg_ctx *c);

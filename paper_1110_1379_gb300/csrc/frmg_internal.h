// frmg_internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>

struct frmg_ctx;

void *frmg_alloc(frmg_ctx *c, size_t bytes);
void frmg_release(frmg_ctx *c, void *p);
void frmg_set_error(const std::string &s);
long long &frmg_launch_counter(frmg_ctx *c);

// abi_guard.h -- keeps C++ exceptions inside the library.
//
// The entry points of the C ABI that use host containers or locks run their body through
// abi_guard.  std::bad_alloc or std::length_error from a container and std::system_error from a
// mutex (all of them host resources running out) become CBESSFM_ERR_OOM with the exception's
// text as the message, so no exception reaches a C caller.  fail() writes into a fixed
// thread-local buffer and cannot throw itself.  A body allocates its host containers before any
// device memory, or frees what it holds on every path, so a caught exception leaks nothing.
#pragma once

#include <exception>

#include "internal.h"

namespace cbessfm {

template <class Body>
cbessfm_status abi_guard(Body&& body) noexcept {
    try {
        return body();
    } catch (const std::exception& ex) {
        return fail(CBESSFM_ERR_OOM, "host resources exhausted: %s", ex.what());
    } catch (...) {
        return fail(CBESSFM_ERR_OOM, "host resources exhausted");
    }
}

}  // namespace cbessfm

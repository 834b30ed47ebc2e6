"""GB300-native minimum distance of binary linear codes (Brouwer-Zimmerman enumeration).

The computation lives in libmdist.so (C-ABI declared in include/mdist.h): host
information-set preparation in C++ and the level enumerator in sm_103a CUDA.  This
package is the Python binding; it loads the library lazily and raises if it is
missing (there is no CPU path).
"""

from .api import Code, device_info, min_distance  # noqa: F401

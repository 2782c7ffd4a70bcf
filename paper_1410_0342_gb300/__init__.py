"""GB300-native GLRM alternating proximal-gradient sweep.

The CUDA library (``libglrm.so``, C ABI declared in ``include/glrm.h``) is
loaded lazily by :mod:`paper_1410_0342_gb300.glrm` so that importing the
package (for example for :mod:`paper_1410_0342_gb300.workloads`) needs no GPU.
"""

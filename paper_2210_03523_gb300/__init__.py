"""GB300-native DGSEM residual, RK3 step and unsteady tau-estimation sweep.

The compute path is the CUDA library ``libdg.so`` behind the C ABI declared
in ``include/dg.h``. ``paper_2210_03523_gb300.dg`` is its thin ctypes
binding. Importing this package loads nothing: ``dg`` loads the library on
first use and raises if it has not been built.
"""

"""GB300-native Parareal fine propagator for 2D Rayleigh-Benard convection.

The compute path is the C-ABI library ``librbc.so`` (CUDA kernels for sm_103a);
``paper_2001_01609_gb300.rbc`` is its thin ctypes binding.  Importing this
package loads nothing; the binding loads the library on first use and raises if
it is missing.  There is no CPU fallback.
"""

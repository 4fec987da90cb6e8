"""GB300-native compact Runge-Kutta Flux Reconstruction (cRKFR) time step.

The compute path is the CUDA library ``libcrkfr.so`` (C ABI declared in
include/cr.h); ``paper_2502_07517_gb300.crkfr`` binds it.  Importing this
package does not load the library; the binding loads it on first use and
raises if it is missing.
"""

"""GB300-native compressible Navier-Stokes right-hand side (WENO5 + Roe + 4th-order viscous
terms) and Runge-Kutta update on a triply periodic grid (arXiv 2211.16718).

The compute path is the C-ABI library ``libns3d.so`` (hand-written CUDA for sm_103a);
``paper_2211_16718_gb300.ns3d`` is its thin Python binding.  Importing this package does
not load the library; the binding loads it on first use and raises if it is missing.
"""
